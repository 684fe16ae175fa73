"""Pins for the oracle's AIM operator (CPU only)."""

import numpy as np
import pytest

from aim_inputs import plate_mesh, icosphere_mesh, random_complex
from oracle import aim
from oracle.efie import dense_Z
from oracle.quadrature import triangle_rule
from oracle.rwg import RWG

K0 = 2 * np.pi
H = 0.1


@pytest.fixture(scope="module")
def plate():
    v, t = plate_mesh(1.0, 9)
    return RWG(v, t)


@pytest.fixture(scope="module")
def ball():
    v, t = icosphere_mesh(0.3, 3)
    return RWG(v, t)


def _integral_g_poly(rwg, m, comp, poly, n=9):
    """int g^c_m p dS with an independent high-order (degree-16) rule."""
    xi1, xi2, w = triangle_rule(n)
    tot = 0.0
    for tri, free, _s, sgn, area in rwg.halves():
        P = rwg.verts[rwg.tris[tri[m]]]
        pts = P[0] + xi1[:, None] * (P[1] - P[0]) + xi2[:, None] * (P[2] - P[0])
        if comp < 3:
            g = sgn * rwg.length[m] / (2 * area[m]) * (pts[:, comp] - rwg.verts[free[m], comp])
        else:
            g = sgn * rwg.length[m] / area[m] * np.ones(len(pts))
        tot += area[m] * np.sum(w * g * poly(pts))
    return tot


@pytest.mark.parametrize("M", [2, 3])
def test_polynomial_reproduction(ball, M):
    """sum_u Lambda_u p(r_u) = int g p for every monomial of per-axis degree <= M."""
    anc = aim.anchors(ball.centre, H, M)
    lam = aim.moment_weights(ball, H, M, anc)
    off = aim.stencil_offsets(M)
    rng = np.random.default_rng(0)
    for m in rng.choice(ball.N, 6, replace=False):
        nodes = H * (anc[m] + off)  # physical node positions
        for q in off:  # exponent triples
            poly = lambda r, q=q: r[..., 0] ** q[0] * r[..., 1] ** q[1] * r[..., 2] ** q[2]
            for c in range(4):
                lhs = np.sum(lam[m, c] * poly(nodes))
                rhs = _integral_g_poly(ball, m, c, poly)
                assert abs(lhs - rhs) <= 1e-13 * max(abs(rhs), 1e-3 * abs(ball.length[m]) * H ** q.sum()) + 1e-15, (m, q, c)


@pytest.mark.parametrize("M", [4, 5])
def test_polynomial_reproduction_high_order(ball, M):
    """Orders 4 and 5 (125 and 216 nodes): the same moment identity with the
    monomials in the stencil's local coordinates (r - h a) / h, where their
    values stay O(1), and the right side from a 10-point rule (the oracle's
    weight rule has 9 points at M = 5); exact to rounding of the sum of the
    terms."""
    anc = aim.anchors(ball.centre, H, M)
    lam = aim.moment_weights(ball, H, M, anc)
    off = aim.stencil_offsets(M)
    rng = np.random.default_rng(1)
    for m in rng.choice(ball.N, 4, replace=False):
        for q in off:
            poly = lambda r, q=q, a=anc[m]: np.prod(((r - H * a) / H) ** q, axis=-1)
            at_nodes = np.prod(off.astype(np.float64) ** q, axis=-1)
            for c in range(4):
                terms = lam[m, c] * at_nodes
                rhs = _integral_g_poly(ball, m, c, poly, n=10)  # degree 18: not the oracle's own rule
                assert abs(terms.sum() - rhs) <= 1e-13 * np.abs(terms).sum() + 1e-16, (m, q, c)


def test_charge_neutral_and_dipole_closed_form(plate):
    anc = aim.anchors(plate.centre, H, 2)
    lam = aim.moment_weights(plate, H, 2, anc)
    v = plate.verts
    assert np.abs(lam[:, 3].sum(-1)).max() <= 1e-14 * np.abs(lam[:, 3]).max()
    cp = v[plate.tris[plate.tri_p]].mean(1)
    cm = v[plate.tris[plate.tri_m]].mean(1)
    dip = 0.5 * plate.length[:, None] * ((cp - v[plate.free_p]) + (v[plate.free_m] - cm))
    assert np.abs(lam[:, :3].sum(-1) - dip).max() <= 1e-15


def test_plate_weights_vanish_off_plane(plate):
    """A z=0 plate anchored at z=-h puts no weight on the z=-h and z=+h planes."""
    anc = aim.anchors(plate.centre, H, 2)
    assert np.all(anc[:, 2] == -1)
    lam = aim.moment_weights(plate, H, 2, anc).reshape(plate.N, 4, 3, 9)
    assert np.abs(lam[:, :, [0, 2], :]).max() <= 1e-15 * np.abs(lam).max()


def test_weights_equal_lagrange_interpolation_moments(ball):
    """Moment solve == int g(r) l_i(xi) l_j(upsilon) l_k(zeta) dS (tensor Lagrange form)."""
    M = 2
    anc = aim.anchors(ball.centre, H, M)
    lam = aim.moment_weights(ball, H, M, anc)
    off = aim.stencil_offsets(M)

    def lag(i, x):
        out = np.ones_like(x)
        for p in range(M + 1):
            if p != i:
                out *= (x - p) / (i - p)
        return out

    for m in (0, 7, ball.N - 1):
        for s, (i, j, k) in enumerate(off):
            poly = lambda r, i=i, j=j, k=k: lag(i, r[..., 0] / H - anc[m, 0]) * lag(j, r[..., 1] / H - anc[m, 1]) * lag(k, r[..., 2] / H - anc[m, 2])
            for c in range(4):
                ref = _integral_g_poly(ball, m, c, poly)
                assert abs(lam[m, c, s] - ref) <= 1e-12 * np.abs(lam[m, c]).max()


def test_anchor_centres_middle_cell(ball):
    anc = aim.anchors(ball.centre, H, 2)
    t = ball.centre / H - anc
    assert np.all(t >= 0.5) and np.all(t < 1.5)


def test_fft_convolution_equals_direct_sum():
    rng = np.random.default_rng(0)
    n = np.array([4, 5, 3])
    Q = rng.standard_normal((2, 3, 5, 4)) + 1j * rng.standard_normal((2, 3, 5, 4))
    for L in ([aim.smooth_length(2 * v - 1) for v in n], [8, 9, 6], [7, 11, 5]):
        L = np.array(L)
        G = aim.green_grid(n, L, H, K0)
        Gh = np.fft.fftn(G)
        got = aim.convolve_fft(Q, Gh, n, L)
        ref = aim.convolve_direct(Q, H, K0)
        assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()
        # Ghat even in each axis
        for ax in range(3):
            flip = np.roll(np.flip(Gh, axis=ax), 1, axis=ax)
            assert np.abs(flip - Gh).max() <= 1e-13 * np.abs(Gh).max()


def test_smooth_length():
    assert [aim.smooth_length(x) for x in (1, 7, 21, 25, 165, 645, 647)] == [1, 8, 24, 25, 180, 648, 648]


def test_near_pairs_brute_force(ball):
    rows, cols = aim.near_pairs(ball.centre, 3 * H)
    c = ball.centre
    d = c[:, None, :] - c[None, :, :]
    d2 = (d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1]) + d[..., 2] * d[..., 2]
    ref = np.argwhere(d2 <= (3 * H) ** 2)
    got = np.stack([rows, cols], 1)
    assert np.array_equal(got, ref)  # argwhere is row-major sorted


def test_gamma_to_infinity_equals_dense(plate):
    """Near radius above the diameter: every pair corrected, Z~ = (Z + Z^T)/2."""
    op = aim.AIMOperator(plate, K0, H, 2, near_radius=10.0)
    Z = dense_Z(plate, K0)
    Zs = 0.5 * (Z + Z.T)
    x = random_complex((3, plate.N), 1)
    y = op.matvec(x)
    ref = x @ Zs.T
    assert np.linalg.norm(y - ref) <= 1e-12 * np.linalg.norm(ref)


def test_symmetry(ball):
    op = aim.AIMOperator(ball, K0, H, 2)
    x = random_complex(ball.N, 2)
    y = random_complex(ball.N, 3)
    a = y @ op.matvec(x)[0]
    b = x @ op.matvec(y)[0]
    assert abs(a - b) <= 1e-13 * abs(a)


def test_diagonal_is_mom_self_term(ball):
    op = aim.AIMOperator(ball, K0, H, 2)
    Z = dense_Z(ball, K0)
    assert np.allclose(op.diagonal(), np.diag(Z), rtol=1e-12, atol=0)
    # and equals the operator's own diagonal
    e = np.zeros((5, ball.N), dtype=complex)
    for i in range(5):
        e[i, 11 * i] = 1
    d = op.matvec(e)[np.arange(5), 11 * np.arange(5)]
    assert np.allclose(d, op.diagonal()[11 * np.arange(5)], rtol=1e-12, atol=0)


def test_error_vs_dense_decreases_with_near_radius(ball):
    """AIM approximation error at gamma = 3, 4, 6 (parity unpinned; recorded, must fall)."""
    Z = dense_Z(ball, K0)
    Zs = 0.5 * (Z + Z.T)
    x = random_complex(ball.N, 4)
    ref = Zs @ x
    errs = []
    for g in (3, 4, 6):
        op = aim.AIMOperator(ball, K0, H, 2, near_radius=g * H)
        errs.append(np.linalg.norm(op.matvec(x)[0] - ref) / np.linalg.norm(ref))
    assert errs[0] < 2e-2
    assert errs[0] > errs[1] > errs[2]


def test_direct_sum_at_nodes_equals_full_direct_sum():
    """convolve_direct_at (sources restricted to the nonzero nodes, outputs to
    listed nodes, chunked) against the all-pairs brute-force sum at every node,
    with a Q that is zero on some nodes of every slice."""
    rng = np.random.default_rng(5)
    Q = rng.standard_normal((2, 3, 5, 4)) + 1j * rng.standard_normal((2, 3, 5, 4))
    Q[:, :, 1, :] = 0.0
    Q[..., 0, 2, 3] = 0.0
    ref = aim.convolve_direct(Q, H, K0)  # [2, 3, 5, 4]
    nz, ny, nx = Q.shape[-3:]
    Z, Y, X = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    nodes = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    for chunk in (7, 1 << 20):  # many chunks and one
        got = aim.convolve_direct_at(Q, nodes, H, K0, chunk=chunk)
        assert np.abs(got - ref.reshape(2, -1)).max() <= 1e-13 * np.abs(ref).max()
    # a few nodes in arbitrary order
    pick = np.array([5, 0, 59, 17])
    got = aim.convolve_direct_at(Q, nodes[pick], H, K0)
    assert np.abs(got - ref.reshape(2, -1)[:, pick]).max() <= 1e-13 * np.abs(ref).max()


@pytest.mark.parametrize("alpha", [1.0, 0.6])
def test_matvec_rows_equals_full_product_rows(ball, alpha):
    """The row-sampled product (direct sum at the rows' stencil nodes) equals
    the FFT product's rows; near list restricted to the rows, EFIE and CFIE."""
    rows = np.array([0, 3, 17, ball.N - 1])
    full = aim.AIMOperator(ball, K0, H, 2, alpha=alpha)
    part = aim.AIMOperator(ball, K0, H, 2, near_rows=rows, alpha=alpha)
    x = random_complex((2, ball.N), 6)
    ref = full.matvec(x)[:, rows]
    got = part.matvec_rows(x, rows)
    assert np.linalg.norm(got - ref) <= 1e-13 * np.linalg.norm(ref)
    assert part._Ghat is None  # the sampled product never builds the padded spectrum


@pytest.mark.parametrize("alpha", [1.0, 0.6])
def test_product_by_components_sums_to_the_product(ball, alpha):
    """Projection, convolution and interpolation run one component at a time
    (comps=[c]) add up to the grid part of the product."""
    op = aim.AIMOperator(ball, K0, H, 2, alpha=alpha)
    x = random_complex((2, ball.N), 8)
    ref = op.far_matvec(x)
    tot = np.zeros_like(ref)
    for c in range(4):
        tot += op.interpolate(op.convolve(op.project(x, comps=[c])), comps=[c])
    assert np.linalg.norm(tot - ref) <= 1e-14 * np.linalg.norm(ref)
    assert np.array_equal(op.project(x, comps=[2])[:, 0], op.project(x)[:, 2])
