"""Pins for the oracle's solver, far field, Mie series and eq. (1) (CPU only)."""

import numpy as np
import pytest

from aim_inputs import plate_mesh, icosphere_mesh, planewave_minus_z_xpol, random_complex
from oracle import aim, mie, rcs, solve
from oracle.efie import dense_Z
from oracle.excitation import planewave_rhs
from oracle.rwg import RWG

K0 = 2 * np.pi
H = 0.1


def test_gmres_matches_lu_on_plate():
    v, t = plate_mesh(1.0, 9)
    r = RWG(v, t)
    op = aim.AIMOperator(r, K0, H, 2)
    kh, p = planewave_minus_z_xpol()
    V = planewave_rhs(r, K0, kh, p)[0]
    Zt = op.matvec(np.eye(r.N)).T  # dense copy of the AIM operator
    x_lu = np.linalg.solve(Zt, V)
    x, it, res = solve.gmres(lambda z: op.matvec(z)[0], V, op.diagonal(), tol=1e-8, restart=50)
    assert res <= 1e-8
    assert np.linalg.norm(x - x_lu) <= 1e-5 * np.linalg.norm(x_lu)


def test_gmres_small_restart_and_exact_system():
    rng = np.random.default_rng(3)
    A = np.eye(40) * 4 + rng.standard_normal((40, 40)) * 0.3 + 1j * rng.standard_normal((40, 40)) * 0.3
    b = rng.standard_normal(40) + 0j
    x, it, res = solve.gmres(lambda z: A @ z, b, np.diag(A), tol=1e-12, restart=7)
    assert np.linalg.norm(A @ x - b) <= 1e-11 * np.linalg.norm(b)


def test_mie_invariants():
    for x in (0.3, 2.0, 25.0):
        qext, qsca, _ = mie.efficiencies(x)
        assert abs(qext - qsca) <= 1e-12 * qsca  # lossless PEC: extinction = scattering
    _, _, qb = mie.efficiencies(0.05)
    assert abs(qb - 9 * 0.05 ** 4) <= 0.01 * 9 * 0.05 ** 4  # Rayleigh limit 9 (ka)^4
    _, _, qb = mie.efficiencies(100.0)
    assert abs(qb - 1.0) < 2e-3  # geometric-optics limit


def test_mie_bistatic_integrates_to_csca():
    """int sigma_tot dOmega / 4 pi from S1, S2 equals C_sca from the coefficient sum."""
    R = 0.7
    x = K0 * R
    th, ph, w = rcs.direction_grid(80, 160)
    S1, S2 = mie.amplitudes(x, th)
    sig = (1.0 / np.pi) * (np.abs(S2) ** 2 * np.cos(ph) ** 2 + np.abs(S1) ** 2 * np.sin(ph) ** 2)
    csca = (sig * w).sum() / (4 * np.pi)
    _, qsca, _ = mie.efficiencies(x)
    assert abs(csca - qsca * np.pi * R ** 2) <= 1e-10 * csca
    # backscatter from the amplitudes equals the coefficient series
    S1b, S2b = mie.amplitudes(x, np.array([np.pi]))
    _, _, qb = mie.efficiencies(x)
    assert abs(4 * np.abs(S1b[0]) ** 2 / x ** 2 - qb) <= 1e-10 * qb


def test_err_thth_eq1_properties():
    th, ph, w = rcs.direction_grid(16, 32)
    s = 1.0 + np.cos(th) ** 2
    assert rcs.err_thth(s, s, w) == 0.0
    assert abs(rcs.err_thth(1.01 * s, s, w) - 0.01) < 1e-14
    assert abs(w.sum() - 4 * np.pi) < 1e-12


@pytest.mark.slow
def test_mom_sphere_rcs_matches_mie():
    """Dense EFIE MoM of a 0.5 lambda PEC sphere (lambda/9 mesh) is within 2.5 % of Mie."""
    from aim_inputs import icosphere_frequency

    R = 0.5
    v, t = icosphere_mesh(R, icosphere_frequency(R))
    r = RWG(v, t)
    Z = dense_Z(r, K0)
    kh, p = planewave_minus_z_xpol()
    V = planewave_rhs(r, K0, kh, p)[0]
    x = solve.lu_solve(0.5 * (Z + Z.T), V)[0]
    n = rcs.default_ntheta(K0 * R)
    th, ph, w = rcs.direction_grid(n, 2 * n)
    s = rcs.sigma_thth(r, K0, x, th, ph)[0]
    ref = mie.sigma_thth_minus_z(R, th, ph)
    e = rcs.err_thth(s, ref, w)
    assert e < 0.025
    # a mirrored pattern (wrong travel direction) is far off
    ref_wrong = mie.sigma_thth_minus_z(R, np.pi - th, ph)
    assert rcs.err_thth(s, ref_wrong, w) > 5 * e


def test_planewave_rhs_closed_form_at_normal_incidence():
    """On the z = 0 plate a wave travelling -z has unit phase everywhere, so
    V_m = pol . int f_m dS, and for an RWG function int f_m dS = (l_m / 3)(p_- - p_+)
    with p_+- the free vertices of its two triangles (the centroid of each
    triangle lies a third of the way from the free vertex to the edge)."""
    v, t = plate_mesh(1.0, 5)
    r = RWG(v, t)
    closed = (r.length / 3.0)[:, None] * (r.verts[r.free_m] - r.verts[r.free_p])
    kz = np.array([[0.0, 0.0, -1.0], [0.0, 0.0, -1.0]])
    pols = np.array([[1.0, 0.0, 0.0], [0.0, 1.0, 0.0]])
    V = planewave_rhs(r, K0, kz, pols)
    assert np.abs(V.imag).max() <= 1e-15 * np.abs(V).max()
    assert np.abs(V.real - (closed @ pols.T).T).max() <= 1e-14 * np.abs(closed).max()
