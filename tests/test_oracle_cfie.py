"""Pins of the oracle's MFIE / CFIE (Section 2.2: CFIE with alpha = 0.6 for closed bodies)."""

import numpy as np
import pytest
import scipy.linalg

from aim_inputs import icosphere_mesh, plate_mesh, planewave_minus_z_xpol, random_incidence
from oracle import ETA0, aim, mfie, mie, rcs
from oracle.efie import dense_Z
from oracle.excitation import planewave_rhs
from oracle.quadrature import triangle_rule
from oracle.rwg import RWG

K0 = 2 * np.pi
H = 0.1


@pytest.fixture(scope="module")
def small_sphere():
    v, t = icosphere_mesh(0.25, 4)
    return RWG(v, t)


def test_mfie_reduces_to_half_gram_on_a_plate():
    """Every pair of a flat plate is coplanar, so n x (grad G x f) vanishes and
    ZM = <f_m, f_n> / 2; the Gram matrix comes from an independent 6-point rule."""
    v, t = plate_mesh(0.5, 4)
    r = RWG(v, t)
    ZM = mfie.dense_ZM(r, K0)
    x1, x2, w = triangle_rule(6)
    G = np.zeros((r.N, r.N))
    for tri_m, free_m, _s, sg_m, area_m in r.halves():
        for tri_n, free_n, _s2, sg_n, area_n in r.halves():
            same = tri_m[:, None] == tri_n[None, :]
            mi, ni = np.nonzero(same)
            for m, n in zip(mi, ni):
                P = r.verts[r.tris[tri_m[m]]]
                pts = P[0] + x1[:, None] * (P[1] - P[0]) + x2[:, None] * (P[2] - P[0])
                fm = sg_m * r.length[m] / (2 * area_m[m]) * (pts - r.verts[free_m[m]])
                fn = sg_n * r.length[n] / (2 * area_n[n]) * (pts - r.verts[free_n[n]])
                G[m, n] += area_m[m] * np.sum(w * (fm * fn).sum(-1))
    assert np.abs(ZM.imag).max() == 0.0
    assert np.abs(ZM.real - 0.5 * G).max() <= 1e-14 * np.abs(G).max()


@pytest.mark.parametrize("M", [2, 3, 4, 5])
def test_mfie_weights_reproduce_the_curl_moments(small_sphere, M):
    """sum_u W^c_m(u) q(u) = int f_m . (n x (grad q x e_c)) dS for every monomial q of
    per-axis degree <= M (local coordinates), right side from a 10-point rule."""
    r = small_sphere
    anc = aim.anchors(r.centre, H, M)
    W = mfie.mfie_weights(r, H, M, anc)
    off = aim.stencil_offsets(M)
    nrm = mfie.tri_normals(r.verts, r.tris)
    x1, x2, w = triangle_rule(10)
    rng = np.random.default_rng(3)
    for m in rng.choice(r.N, 4, replace=False):
        for q in off[rng.choice(len(off), 8, replace=False)]:
            at_nodes = np.prod(off.astype(np.float64) ** q, axis=-1)
            rhs = np.zeros(3)
            for tri, free, _s, sg, area in r.halves():
                P = r.verts[r.tris[tri[m]]]
                pts = P[0] + x1[:, None] * (P[1] - P[0]) + x2[:, None] * (P[2] - P[0])
                f = sg * r.length[m] / (2 * area[m]) * (pts - r.verts[free[m]])
                loc = (pts - H * anc[m]) / H
                grad = np.zeros_like(loc)
                for d in range(3):
                    g = np.ones(len(loc))
                    for e in range(3):
                        g = g * (q[e] * loc[:, e] ** (q[e] - 1) if e == d and q[e] > 0 else
                                 (np.zeros(len(loc)) if e == d else loc[:, e] ** q[e]))
                    grad[:, d] = g / H
                n = nrm[tri[m]]
                for c in range(3):
                    integrand = (f * grad).sum(-1) * n[c] - f[:, c] * (grad @ n)
                    rhs[c] += area[m] * np.sum(w * integrand)
            for c in range(3):
                terms = W[m, c] * at_nodes
                assert abs(terms.sum() - rhs[c]) <= 1e-12 * (np.abs(terms).sum() + abs(rhs[c])) + 1e-16, (m, q, c)


def test_cfie_all_pairs_near_equals_dense(small_sphere):
    """Near radius beyond the body: the AIM CFIE operator is the dense CFIE matrix
    (EFIE part symmetrised), diagonal included."""
    r = small_sphere
    alpha = 0.6
    ZE = dense_Z(r, K0)
    ZC = alpha * 0.5 * (ZE + ZE.T) + (1 - alpha) * ETA0 * mfie.dense_ZM(r, K0)
    op = aim.AIMOperator(r, K0, H, 2, near_radius=10.0, alpha=alpha)
    x = np.random.default_rng(0).normal(size=(2, r.N)) + 1j * np.random.default_rng(1).normal(size=(2, r.N))
    y = op.matvec(x)
    ref = (ZC @ x.T).T
    assert np.linalg.norm(y - ref) <= 1e-12 * np.linalg.norm(ref)
    assert np.abs(op.diagonal() - np.diag(ZC)).max() <= 1e-12 * np.abs(np.diag(ZC)).max()


def test_cfie_sphere_rcs_near_mie_and_better_conditioned(small_sphere):
    """Dense CFIE (alpha = 0.6) solution of a 0.25 lambda sphere: bistatic RCS within a few
    percent of Mie (coarse mesh), close to the EFIE solution's, and a far smaller
    condition number than the EFIE matrix."""
    r = small_sphere
    ZE = dense_Z(r, K0)
    ZES = 0.5 * (ZE + ZE.T)
    ZM = mfie.dense_ZM(r, K0)
    kh, po = planewave_minus_z_xpol()
    VE = planewave_rhs(r, K0, kh, po)[0]
    VC = mfie.planewave_rhs_cfie(r, K0, kh, po, 0.6)[0]
    ZC = 0.6 * ZES + 0.4 * ETA0 * ZM
    xe = scipy.linalg.solve(ZES, VE)
    xc = scipy.linalg.solve(ZC, VC)
    n = rcs.default_ntheta(K0 * 0.25)
    th, ph, w = rcs.direction_grid(n, 2 * n)
    ref = mie.sigma_thth_minus_z(0.25, th, ph)
    se = rcs.sigma_thth(r, K0, xe[None], th, ph)[0]
    sc = rcs.sigma_thth(r, K0, xc[None], th, ph)[0]
    assert rcs.err_thth(sc, ref, w) < 0.06
    assert rcs.err_thth(sc, se, w) < 0.05
    assert np.linalg.cond(ZC) < 0.5 * np.linalg.cond(ZES)


def test_mfie_rhs_on_a_plate_reduces_to_efie_moments():
    """On a flat plate with unit normal n, n x (khat x pol) = khat (n . pol) - pol (n . khat)
    is a constant vector, so eta V^M = (n . pol) <f, khat e> - (n . khat) <f, pol e>: two
    EFIE-type moments of the same phase (the EFIE right-hand side evaluated with khat and
    with pol as the polarisation).  At normal incidence from above (khat = -z, pol = x,
    n = +z) this is exactly V^E."""
    v, t = plate_mesh(1.0, 6)
    r = RWG(v, t)
    nz = mfie.tri_normals(r.verts, r.tris)
    assert np.allclose(np.abs(nz[:, 2]), 1.0)
    n = nz[0]
    assert np.all(nz == n)  # one orientation over the plate
    kh, po = random_incidence(3, seed=11)
    VM = ETA0 * mfie.planewave_rhs_mfie(r, K0, kh, po)
    ref = (po @ n)[:, None] * planewave_rhs(r, K0, kh, kh) - (kh @ n)[:, None] * planewave_rhs(r, K0, kh, po)
    assert np.linalg.norm(VM - ref) <= 1e-13 * np.linalg.norm(ref)
    kz, px = np.array([[0.0, 0.0, -1.0]]), np.array([[1.0, 0.0, 0.0]])
    VMn = ETA0 * mfie.planewave_rhs_mfie(r, K0, kz, px)
    VEn = planewave_rhs(r, K0, kz, px)
    assert np.linalg.norm(VMn - n[2] * VEn) <= 1e-13 * np.linalg.norm(VEn)


def test_mfie_alone_reproduces_mie(small_sphere):
    """The MFIE by itself (alpha = 0: ZM x = VM) on the 0.25 lambda sphere gives a
    bistatic RCS within 6 % of the Mie series: the identity term, the sign and the
    orientation of the n x grad G x f term and the n x H_inc excitation all enter
    this solution without the EFIE's help."""
    r = small_sphere
    ZM = mfie.dense_ZM(r, K0)
    kh, po = planewave_minus_z_xpol()
    VM = mfie.planewave_rhs_mfie(r, K0, kh, po)[0]
    x = scipy.linalg.solve(ZM, VM)
    n = rcs.default_ntheta(K0 * 0.25)
    th, ph, w = rcs.direction_grid(n, 2 * n)
    s = rcs.sigma_thth(r, K0, x[None], th, ph)[0]
    assert rcs.err_thth(s, mie.sigma_thth_minus_z(0.25, th, ph), w) < 0.06
    # the same solve with the second term's sign flipped is far off
    Zbad = ZM - 2.0 * (ZM - 0.5 * _gram(r))
    xb = scipy.linalg.solve(Zbad, VM)
    sb = rcs.sigma_thth(r, K0, xb[None], th, ph)[0]
    assert rcs.err_thth(sb, mie.sigma_thth_minus_z(0.25, th, ph), w) > 0.15


def _gram(r):
    """<f_m, f_n> from an independent 6-point rule (equal-triangle halves only)."""
    x1, x2, w = triangle_rule(6)
    G = np.zeros((r.N, r.N))
    halves = list(r.halves())
    for tri_m, free_m, _s, sg_m, area_m in halves:
        for tri_n, free_n, _s2, sg_n, area_n in halves:
            mi, ni = np.nonzero(tri_m[:, None] == tri_n[None, :])
            for m, n in zip(mi, ni):
                P = r.verts[r.tris[tri_m[m]]]
                pts = P[0] + x1[:, None] * (P[1] - P[0]) + x2[:, None] * (P[2] - P[0])
                fm = sg_m * r.length[m] / (2 * area_m[m]) * (pts - r.verts[free_m[m]])
                fn = sg_n * r.length[n] / (2 * area_n[n]) * (pts - r.verts[free_n[n]])
                G[m, n] += area_m[m] * np.sum(w * (fm * fn).sum(-1))
    return G
