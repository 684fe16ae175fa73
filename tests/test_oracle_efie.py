"""Pins for the oracle's EFIE entries (CPU only)."""

import numpy as np
import pytest
from scipy import integrate

from aim_inputs import plate_mesh, icosphere_mesh, random_complex
from oracle import ETA0
from oracle.efie import potential_integrals, _smooth_kernel, dense_Z, triangle_pair_blocks, mom_entries
from oracle.rcs import far_field, direction_grid
from oracle.rwg import RWG

TRI = np.array([[0.1, -0.05, 0.2], [0.35, 0.02, 0.25], [0.12, 0.3, 0.1]])


def _adaptive(fun, tv):
    """int_T fun(r') dS' by nested adaptive Gauss-Kronrod on the collapsed square."""
    r0, r1, r2 = tv
    A2 = np.linalg.norm(np.cross(r1 - r0, r2 - r0))

    def f(t, s):
        rp = r0 + s * (r1 - r0) + t * (1.0 - s) * (r2 - r0)
        return fun(rp) * A2 * (1.0 - s)

    val, err = integrate.dblquad(f, 0.0, 1.0, 0.0, 1.0, epsabs=1e-14, epsrel=1e-13)
    return val


@pytest.mark.parametrize("h", [0.3, 0.05, -0.02])
@pytest.mark.parametrize("where", [(0.2, 0.1), (0.5, 0.6), (-0.1, 0.05)])
def test_potential_integrals_vs_adaptive(h, where):
    """Closed-form int 1/R and int (rho'-rho)/R vs adaptive quadrature (<= 1e-10)."""
    r0, r1, r2 = TRI
    n = np.cross(r1 - r0, r2 - r0)
    n /= np.linalg.norm(n)
    r = r0 + where[0] * (r1 - r0) + where[1] * (r2 - r0) + h * n
    I0, I1, rho = potential_integrals(r[None], TRI[None])
    ref0 = _adaptive(lambda rp: 1.0 / np.linalg.norm(r - rp), TRI)
    assert abs(I0[0] - ref0) <= 1e-10 * abs(ref0)
    for c in range(3):
        ref = _adaptive(lambda rp: (rp - rho[0])[c] / np.linalg.norm(r - rp), TRI)
        assert abs(I1[0, c] - ref) <= 1e-10 * max(abs(ref0), 1.0) * 0.1 + 1e-12


def test_potential_in_plane_outside_on_edge_line():
    """In-plane observation points, including one on an edge's extension line."""
    r0, r1, r2 = TRI
    for r in (r0 + 1.3 * (r1 - r0) + 0.0 * (r2 - r0), r0 - 0.4 * (r1 - r0) - 0.3 * (r2 - r0)):
        I0, I1, rho = potential_integrals(r[None], TRI[None])
        ref0 = _adaptive(lambda rp: 1.0 / np.linalg.norm(r - rp), TRI)
        assert abs(I0[0] - ref0) <= 1e-10 * abs(ref0)


def test_potential_self_centroid_closed_form():
    """Equilateral triangle, observer at the centroid: int 1/R = 3 h ln(tan(pi/3)+sec(pi/3)) ... ."""
    a = 0.2
    tv = np.array([[0, 0, 0], [a, 0, 0], [a / 2, a * np.sqrt(3) / 2, 0]], dtype=float)
    c = tv.mean(0)
    I0, _, _ = potential_integrals(c[None], tv[None])
    # distance to each edge d = a / (2 sqrt 3); each edge subtends +-pi/3 from c:
    # int over one sub-triangle = d * ln(tan(pi/4 + t/2)) from -pi/3 to pi/3
    d = a / (2 * np.sqrt(3))
    exact = 3 * d * 2 * np.log(np.tan(np.pi / 4 + np.pi / 6))
    assert abs(I0[0] - exact) < 1e-14


def test_smooth_kernel_matches_direct():
    k = 2 * np.pi
    R = np.array([1e-3, 0.01, 0.1, 0.7])
    direct = (np.exp(-1j * k * R) - 1.0) / (4 * np.pi * R)
    assert np.allclose(_smooth_kernel(k, R), direct, rtol=1e-12, atol=0)
    assert np.allclose(_smooth_kernel(k, np.array([0.0])), -1j * k / (4 * np.pi))


def test_singular_extraction_matches_brute_force_far_pair():
    """For triangles sharing no vertex the split and unsplit kernels agree."""
    v, t = plate_mesh(1.0, 6)
    k = 2 * np.pi
    P = np.array([0, 0])
    Q = np.array([30, 30])
    a = triangle_pair_blocks(v, t, P[:1], Q[:1], k, singular=np.array([False]), n_src=10, n_test_sing=3)
    b = triangle_pair_blocks(v, t, P[:1], Q[:1], k, singular=np.array([True]), n_src=10, n_test_sing=3)
    assert np.abs(a - b).max() <= 1e-8 * np.abs(a).max()


def test_self_term_converges_with_rule_order():
    """Quadrature-order convergence of a coincident-triangle block."""
    v, t = plate_mesh(1.0, 9)
    k = 2 * np.pi
    vals = [triangle_pair_blocks(v, t, [3], [3], k, n_test=nt, n_src=ns, n_test_sing=nt)[0, 0, 0]
            for nt, ns in ((3, 4), (5, 6), (8, 8), (12, 12), (20, 20))]
    errs = [abs(x - vals[-1]) for x in vals[:-1]]
    assert errs[0] > errs[1] > errs[2] > errs[3]
    assert errs[0] < 1e-2 * abs(vals[-1])  # the default rules: within 1 %
    assert errs[3] < 1e-4 * abs(vals[-1])


def test_galerkin_symmetry_before_symmetrisation():
    v, t = plate_mesh(1.0, 4)
    r = RWG(v, t)
    Z = dense_Z(r, 2 * np.pi)
    assert np.abs(Z - Z.T).max() <= 2e-3 * np.abs(Z).max()
    assert np.abs(Z - Z.T).max() > 0  # the two orders use different rules


def test_mom_entries_match_dense():
    v, t = plate_mesh(1.0, 4)
    r = RWG(v, t)
    k = 2 * np.pi
    Z = dense_Z(r, k)
    rng = np.random.default_rng(1)
    rows = rng.integers(0, r.N, 40)
    cols = rng.integers(0, r.N, 40)
    z = mom_entries(r, rows, cols, k)
    assert np.allclose(z, Z[rows, cols], rtol=1e-13, atol=0)


def test_radiated_power_identity():
    """(k^2 eta / 32 pi^2) int |N_perp|^2 dOmega = Re(x^H Z x) / 2 for any current x.

    Re Z is the radiation (sin kR / R) part of the EFIE kernel, so the
    far-field power of a current equals half the real part of its quadratic
    form: pins the far-field normalisation against Z.
    """
    v, t = icosphere_mesh(0.3, 3)
    r = RWG(v, t)
    k = 2 * np.pi
    Z = dense_Z(r, k)
    Zs = 0.5 * (Z + Z.T)
    x = random_complex(r.N, 5)
    th, ph, w = direction_grid(48, 96)
    Nt, Np = far_field(r, k, x, th, ph)
    prad = k * k * ETA0 / (32 * np.pi ** 2) * ((np.abs(Nt[0]) ** 2 + np.abs(Np[0]) ** 2) * w).sum()
    quad = 0.5 * np.real(np.vdot(x, Zs @ x))
    assert abs(prad - quad) <= 5e-3 * abs(quad)
