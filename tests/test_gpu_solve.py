"""GPU solver and RCS against the oracle (through the C ABI).

Gates: true relative residual <= 1e-6 for the plain complex128 solve and for
the complex64 solve with FP64 refinement; RCS parity 1e-6; err_thth of the
mixed solve <= err_thth of the plain solve + 1e-3 (eq. 1 against Mie).
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from aim_inputs import icosphere_frequency, icosphere_mesh, plate_mesh, planewave_minus_z_xpol, random_incidence  # noqa: E402
from oracle import aim as oaim, mie, rcs as orcs, solve as osolve  # noqa: E402
from oracle.excitation import planewave_rhs  # noqa: E402
from oracle.rwg import RWG  # noqa: E402

import paper_1010_1456_gb300 as g  # noqa: E402

K0 = 2 * np.pi
H = 0.1
TOL = 1e-6


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


@pytest.fixture(scope="module")
def sphere():
    R = 0.5
    v, t = icosphere_mesh(R, icosphere_frequency(R))
    op = oaim.AIMOperator(RWG(v, t), K0, H, 2)
    return R, v, t, op


def true_res(op, V, X):
    return np.linalg.norm(V - op.matvec(X), axis=1) / np.linalg.norm(V, axis=1)


@pytest.mark.parametrize("prec", [g.AIM_C128, g.AIM_C128_F64, g.AIM_C64])
def test_solve_plate_reaches_tolerance(prec):
    v, t = plate_mesh(1.0, 9)
    op = oaim.AIMOperator(RWG(v, t), K0, H, 2)
    ctx = g.aim_setup(v, t, K0, H, precision=prec)
    kh, po = planewave_minus_z_xpol()
    V = g.aim_rhs_planewave(ctx, kh, po)
    X, info = g.aim_solve(ctx, V, TOL)
    assert info["converged"].all() and info["rel_res"].max() <= TOL
    Vn, Xn = V.cpu().numpy(), X.cpu().numpy()
    assert true_res(op, Vn, Xn).max() <= 1.01 * TOL
    xo, it, res = osolve.gmres(lambda z: op.matvec(z)[0], Vn[0], op.diagonal(), tol=1e-10)
    assert np.linalg.norm(Xn[0] - xo) <= 1e-4 * np.linalg.norm(xo)


def test_multi_rhs_solve_equals_single(sphere):
    R, v, t, op = sphere
    kh, po = random_incidence(2, seed=0)  # 4 right-hand sides
    ctx4 = g.aim_setup(v, t, K0, H, max_rhs=4, precision=g.AIM_C64)
    V = g.aim_rhs_planewave(ctx4, kh, po)
    X4, info = g.aim_solve(ctx4, V, TOL)
    assert info["converged"].all()
    Vn, X4n = V.cpu().numpy(), X4.cpu().numpy()
    assert true_res(op, Vn, X4n).max() <= 1.01 * TOL
    ctx1 = g.aim_setup(v, t, K0, H, max_rhs=1, precision=g.AIM_C64)
    for b in (0, 3):
        X1, _ = g.aim_solve(ctx1, V[b : b + 1].contiguous(), TOL)
        d = np.linalg.norm(X1.cpu().numpy()[0] - X4n[b]) / np.linalg.norm(X4n[b])
        assert d <= 1e-4


def test_rcs_parity_and_mixed_accuracy(sphere):
    R, v, t, op = sphere
    n = orcs.default_ntheta(K0 * R)
    th, ph, w = orcs.direction_grid(n, 2 * n)
    kh, po = planewave_minus_z_xpol()
    errs = {}
    for prec in (g.AIM_C128_F64, g.AIM_C128, g.AIM_C64):
        ctx = g.aim_setup(v, t, K0, H, precision=prec)
        V = g.aim_rhs_planewave(ctx, kh, po)
        X, info = g.aim_solve(ctx, V, TOL)
        stt, spp = g.aim_rcs(ctx, X, th, ph)
        ref = orcs.sigma_thth(op.rwg, K0, X.cpu().numpy(), th, ph)
        assert np.linalg.norm(stt - ref) <= 1e-6 * np.linalg.norm(ref)
        errs[prec] = orcs.err_thth(stt[0], mie.sigma_thth_minus_z(R, th, ph), w)
    assert errs[g.AIM_C64] <= errs[g.AIM_C128_F64] + 1e-3
    assert abs(errs[g.AIM_C128] - errs[g.AIM_C128_F64]) <= 1e-6
    assert errs[g.AIM_C128_F64] < 0.1


def test_zero_rhs_returns_zero():
    v, t = plate_mesh(1.0, 3)
    ctx = g.aim_setup(v, t, K0, H)
    V = torch.zeros((1, ctx.N), dtype=torch.complex128, device="cuda")
    X, info = g.aim_solve(ctx, V, TOL)
    assert info["converged"].all()
    assert torch.count_nonzero(X).item() == 0


def test_iteration_limit_reports_noconv():
    v, t = plate_mesh(1.0, 9)
    ctx = g.aim_setup(v, t, K0, H, maxit=3, restart=3)
    kh, po = planewave_minus_z_xpol()
    V = g.aim_rhs_planewave(ctx, kh, po)
    X, info = g.aim_solve(ctx, V, 1e-12, raise_on_noconv=False)
    assert info["status"] == g.AIM_ENOCONV and not info["converged"].any()
    assert 0 < info["rel_res"][0] < 1.0  # X holds the last iterate, better than zero


def test_graph_replayed_steps_equal_direct_launches(sphere):
    """Arnoldi steps replayed from the captured CUDA graph give the same
    iterate, bit for bit, as the same steps launched one by one (the profiler
    forces direct launches); also on a caller's non-default stream."""
    R, v, t, op = sphere
    kh, po = random_incidence(1, seed=5)  # 2 right-hand sides
    ctx = g.aim_setup(v, t, K0, H, max_rhs=2, precision=g.AIM_C64)
    V = g.aim_rhs_planewave(ctx, kh, po)
    g.aim_solve(ctx, V, TOL)  # one-time allocations and conversions of the first solve
    l0 = g.aim_launch_count(ctx)
    Xg, ig = g.aim_solve(ctx, V, TOL)
    launches_graph = g.aim_launch_count(ctx) - l0
    g.aim_profile(ctx, 1)
    l0 = g.aim_launch_count(ctx)
    Xd, idd = g.aim_solve(ctx, V, TOL)
    launches_direct = g.aim_launch_count(ctx) - l0
    g.aim_profile(ctx, 0)
    assert ig["iterations"] == idd["iterations"] and launches_graph == launches_direct
    assert torch.equal(Xg, Xd)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        g.aim_set_stream(ctx, s)
        Xs, _ = g.aim_solve(ctx, V, TOL)
    s.synchronize()
    g.aim_set_stream(ctx, torch.cuda.current_stream())
    assert torch.equal(Xs, Xg)
    assert true_res(op, V.cpu().numpy(), Xg.cpu().numpy()).max() <= 1.01 * TOL


# ---------------------------------------------------------------- TFQMR
@pytest.mark.parametrize("prec", [g.AIM_C64, g.AIM_C128])
def test_tfqmr_reaches_tolerance_and_matches_gmres(prec):
    """TFQMR (aim_opts.krylov = AIM_TFQMR) on the 1 lambda plate with three
    right-hand sides: every true residual <= 1e-6 against the oracle operator,
    the solutions equal GMRES's to the tolerance."""
    v, t = plate_mesh(1.0, 9)
    op = oaim.AIMOperator(RWG(v, t), K0, H, 2)
    ctx = g.aim_setup(v, t, K0, H, precision=prec, max_rhs=3, krylov=g.AIM_TFQMR)
    kh, po = random_incidence(2, seed=3)
    V = g.aim_rhs_planewave(ctx, kh[:3], po[:3])
    X, info = g.aim_solve(ctx, V, TOL)
    assert info["converged"].all() and info["rel_res"].max() <= TOL
    Vn, Xn = V.cpu().numpy(), X.cpu().numpy()
    assert true_res(op, Vn, Xn).max() <= 1.01 * TOL
    g.aim_set_krylov(ctx, g.AIM_GMRES)
    Xg, ig = g.aim_solve(ctx, V, TOL)
    assert ig["converged"].all()
    Xgn = Xg.cpu().numpy()
    assert np.linalg.norm(Xn - Xgn) <= 1e-4 * np.linalg.norm(Xgn)


def test_tfqmr_cfie_sphere_graph_equals_direct(sphere):
    """TFQMR on the CFIE sphere (alpha 0.6): the step pairs replayed from the
    captured graph give the iterate of direct launches bit for bit, and the
    solution meets the tolerance against the oracle's CFIE operator."""
    R, v, t, _ = sphere
    op = oaim.AIMOperator(RWG(v, t), K0, H, 2, alpha=0.6)
    kh, po = random_incidence(1, seed=8)
    ctx = g.aim_setup(v, t, K0, H, max_rhs=2, precision=g.AIM_C64, cfie_alpha=0.6, krylov=g.AIM_TFQMR)
    V = g.aim_rhs_planewave(ctx, kh, po)
    g.aim_solve(ctx, V, TOL)  # first-solve allocations
    Xg, ig = g.aim_solve(ctx, V, TOL)
    g.aim_profile(ctx, 1)
    Xd, idd = g.aim_solve(ctx, V, TOL)
    g.aim_profile(ctx, 0)
    assert ig["iterations"] == idd["iterations"] and torch.equal(Xg, Xd)
    assert ig["converged"].all()
    assert true_res(op, V.cpu().numpy(), Xg.cpu().numpy()).max() <= 1.01 * TOL


def test_tfqmr_rejects_unknown_method():
    v, t = plate_mesh(1.0, 9)
    with pytest.raises(g.AIMError):
        g.aim_setup(v, t, K0, H, krylov=7)
    ctx = g.aim_setup(v, t, K0, H)
    with pytest.raises(g.AIMError):
        g.aim_set_krylov(ctx, 2)
