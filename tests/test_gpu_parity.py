"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (relative L2 unless stated): complex128 product 1e-12, complex64
product 1e-5, setup arrays 1e-12 (FP64 both sides, different summation
order), right-hand side 1e-12, RCS 1e-6 (the far-field phase factor is taken
in FP32 after an FP64 range reduction).
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from aim_inputs import (  # noqa: E402
    icosphere_frequency,
    icosphere_mesh,
    plate_mesh,
    planewave_minus_z_xpol,
    random_complex,
    random_incidence,
)
from oracle import aim as oaim  # noqa: E402
from oracle.excitation import planewave_rhs  # noqa: E402
from oracle.rwg import RWG  # noqa: E402

import paper_1010_1456_gb300 as g  # noqa: E402

K0 = 2 * np.pi
H = 0.1


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    g.load()


def make(verts, tris, M=2, radius=None, max_rhs=1, precision=g.AIM_C128, near_rows=None, planar=True):
    r = 3 * H if radius is None else radius
    ctx = g.aim_setup(verts, tris, K0, H, M=M, near_radius=r, max_rhs=max_rhs, precision=precision, planar=planar)
    op = oaim.AIMOperator(RWG(verts, tris), K0, H, M, near_radius=r, near_rows=near_rows)
    return ctx, op


@pytest.fixture(scope="module")
def plate_a():
    """1 lambda plate on the full three-dimensional grid (no plane collapse)."""
    v, t = plate_mesh(1.0, 9)
    return make(v, t, max_rhs=3, planar=False)


@pytest.fixture(scope="module")
def plate_a_planar():
    """The same plate with its grid collapsed to the z = 0 plane."""
    v, t = plate_mesh(1.0, 9)
    return make(v, t, max_rhs=17)


@pytest.fixture(scope="module")
def sphere_small():
    R = 0.5
    v, t = icosphere_mesh(R, icosphere_frequency(R))
    return make(v, t, max_rhs=2)


def test_setup_arrays_match_oracle(plate_a):
    ctx, op = plate_a
    assert ctx.N == op.N == 225
    n, L, nnz = g.aim_grid_info(ctx)
    assert n == list(op.n) and L == list(op.L)
    assert np.array_equal(g.aim_export(ctx, g.AIM_EXPORT_ANCHORS), op.anc)
    lam = g.aim_export(ctx, g.AIM_EXPORT_WEIGHTS)
    assert np.abs(lam - op.lam).max() <= 1e-12 * np.abs(op.lam).max()
    ptr = g.aim_export(ctx, g.AIM_EXPORT_NEAR_PTR)
    col = g.aim_export(ctx, g.AIM_EXPORT_NEAR_COL)
    assert nnz == len(op.near_rows)
    assert np.array_equal(np.repeat(np.arange(ctx.N), np.diff(ptr)), op.near_rows)
    assert np.array_equal(col, op.near_cols)
    val = g.aim_export(ctx, g.AIM_EXPORT_NEAR_VAL)
    assert rel(val, op.near_vals) <= 1e-12
    assert rel(g.aim_export(ctx, g.AIM_EXPORT_DIAG), op.diagonal()) <= 1e-12
    gh = g.aim_export(ctx, g.AIM_EXPORT_GHAT)
    ref = op.Ghat[: L[2] // 2 + 1, : L[1] // 2 + 1, : L[0] // 2 + 1] / np.prod(L)
    assert rel(gh, ref) <= 1e-13


WIDE = [g.AIM_C128, g.AIM_C128_F64]  # float-float FFT and native FP64


@pytest.mark.parametrize("prec", WIDE)
@pytest.mark.parametrize("nrhs", [1, 3])
def test_matvec_c128_plate(plate_a, nrhs, prec):
    ctx, op = plate_a
    x = random_complex((nrhs, ctx.N), 11)
    y = g.aim_matvec(ctx, torch.from_numpy(x).cuda(), precision=prec).cpu().numpy()
    assert rel(y, op.matvec(x)) <= 1e-12


def test_matvec_c64_plate(plate_a):
    ctx, op = plate_a
    x = random_complex((3, ctx.N), 12)
    y = g.aim_matvec(ctx, torch.from_numpy(x.astype(np.complex64)).cuda()).cpu().numpy()
    assert rel(y, op.matvec(x.astype(np.complex64).astype(np.complex128))) <= 1e-5


def test_matvec_sphere_all_precisions(sphere_small):
    ctx, op = sphere_small
    x = random_complex((2, ctx.N), 13)
    ref = op.matvec(x)
    for prec in WIDE:
        y = g.aim_matvec(ctx, torch.from_numpy(x).cuda(), precision=prec).cpu().numpy()
        assert rel(y, ref) <= 1e-12
    y32 = g.aim_matvec(ctx, torch.from_numpy(x.astype(np.complex64)).cuda()).cpu().numpy()
    assert rel(y32, ref) <= 1e-5


def test_matvec_host_entry_point(plate_a):
    ctx, op = plate_a
    x = random_complex((2, ctx.N), 14)
    for prec in WIDE:
        assert rel(g.aim_matvec_host(ctx, x, precision=prec), op.matvec(x)) <= 1e-12
    y32 = g.aim_matvec_host(ctx, x.astype(np.complex64), precision=g.AIM_C64)
    assert rel(y32, op.matvec(x.astype(np.complex64).astype(np.complex128))) <= 1e-5
    # pinned torch host buffers give the same bytes
    xp = torch.from_numpy(x).pin_memory()
    yp = torch.empty_like(xp).pin_memory()
    g.aim_matvec_host(ctx, xp, precision=g.AIM_C128, out=yp)
    assert np.array_equal(yp.numpy(), g.aim_matvec_host(ctx, x, precision=g.AIM_C128))


def test_rhs_matches_oracle(sphere_small):
    ctx, op = sphere_small
    kh, po = random_incidence(1, seed=3)
    V = g.aim_rhs_planewave(ctx, kh, po).cpu().numpy()
    assert rel(V, planewave_rhs(op.rwg, K0, kh, po)) <= 1e-12


@pytest.mark.parametrize("M", [1, 3, 4, 5])
def test_other_stencil_orders(M):
    """Orders 1 to 5 (8 to 216 stencil nodes), both FP64-accurate products."""
    v, t = plate_mesh(0.7, 6)
    ctx, op = make(v, t, M=M)
    x = random_complex((1, ctx.N), 15)
    ref = op.matvec(x)
    for prec in WIDE:
        y = g.aim_matvec(ctx, torch.from_numpy(x).cuda(), precision=prec).cpu().numpy()
        assert rel(y, ref) <= 1e-12, (prec, rel(y, ref))


@pytest.mark.parametrize("planar", [True, False])
@pytest.mark.parametrize("nrhs", [8, 9, 17, 65, 70])
def test_many_rhs_products(nrhs, planar):
    """Batches of 8 to 70 right-hand sides (lanes, tiles and grid chunks cover every RHS),
    on the plate's collapsed and full grids."""
    v, t = plate_mesh(1.0, 9)
    ctx, op = make(v, t, max_rhs=nrhs, planar=planar)
    x = random_complex((nrhs, ctx.N), 40 + nrhs)
    ref = op.matvec(x)
    for prec in WIDE:
        y = g.aim_matvec(ctx, torch.from_numpy(x).cuda(), precision=prec).cpu().numpy()
        assert rel(y, ref) <= 1e-12
    y32 = g.aim_matvec(ctx, torch.from_numpy(x.astype(np.complex64)).cuda()).cpu().numpy()
    assert rel(y32, op.matvec(x.astype(np.complex64).astype(np.complex128))) <= 1e-5
    # each right-hand side on its own equals its column of the batch
    for b in (0, nrhs - 1):
        yb = g.aim_matvec(ctx, torch.from_numpy(x[b : b + 1]).cuda(), precision=g.AIM_C128).cpu().numpy()
        assert rel(yb[0], ref[b]) <= 1e-12


def test_group_projection_across_batch_sizes():
    """A sphere's grid has z passes, so the projection writes only the 8-node
    groups that hold entries, and the rest of the projection grid keeps the
    zeros written when the grids were allocated.  Batches of 3, then 17 (the
    many-RHS projection, which writes every node), then 3 and 1 right-hand
    sides, in every precision, match the oracle."""
    R = 0.5
    v, t = icosphere_mesh(R, icosphere_frequency(R))
    ctx, op = make(v, t, max_rhs=17)
    for nrhs in (3, 17, 3, 1):
        x = random_complex((nrhs, ctx.N), 60 + nrhs)
        ref = op.matvec(x)
        for prec in WIDE:
            y = g.aim_matvec(ctx, torch.from_numpy(x).cuda(), precision=prec).cpu().numpy()
            assert rel(y, ref) <= 1e-12, (nrhs, prec)
        y32 = g.aim_matvec(ctx, torch.from_numpy(x.astype(np.complex64)).cuda()).cpu().numpy()
        assert rel(y32, op.matvec(x.astype(np.complex64).astype(np.complex128))) <= 1e-5, nrhs


FFT_CHOICES = [g.AIM_FFT_STOCKHAM, g.AIM_FFT_FOURSTEP, g.AIM_FFT_FOURSTEP_SMALL, g.AIM_FFT_FOURSTEP_WARP,
               g.AIM_FFT_FOURSTEP_WIDE]


@pytest.mark.parametrize("kernel", FFT_CHOICES)
def test_every_fft_kernel_choice(plate_a, plate_a_planar, sphere_small, kernel):
    """Each FFT kernel, forced on all five passes, gives the oracle's product in every precision."""
    for (ctx, op), nrhs, seed in ((plate_a, 3, 31), (plate_a_planar, 3, 34), (sphere_small, 2, 32)):
        x = random_complex((nrhs, ctx.N), seed)
        ref = op.matvec(x)
        for prec in WIDE + [g.AIM_C64]:
            assert g.aim_fft_config(ctx, prec, [kernel] * 5) == [kernel] * 5
            xt = torch.from_numpy(x if prec != g.AIM_C64 else x.astype(np.complex64)).cuda()
            y = g.aim_matvec(ctx, xt, precision=prec).cpu().numpy()
            if prec == g.AIM_C64:
                assert rel(y, op.matvec(x.astype(np.complex64).astype(np.complex128))) <= 1e-5
            else:
                assert rel(y, ref) <= 1e-12
            g.aim_fft_config(ctx, prec, [g.AIM_FFT_AUTO] * 5)


def test_autotune_keeps_parity_and_profiler_state(sphere_small):
    ctx, op = sphere_small
    x = random_complex((2, ctx.N), 33)
    xt = torch.from_numpy(x).cuda()
    g.aim_profile(ctx, 2)
    g.aim_profile(ctx, 1)
    g.aim_matvec(ctx, xt, precision=g.AIM_C128)
    before = g.aim_profile_read(ctx)
    kernels, ms = g.aim_autotune(ctx, g.AIM_C128, nrhs=2, reps=2)
    after = g.aim_profile_read(ctx)
    g.aim_profile(ctx, 0)
    g.aim_profile(ctx, 2)
    assert {k: v[0] for k, v in after.items()} == {k: v[0] for k, v in before.items()}
    assert all(k in FFT_CHOICES for k in kernels)
    assert g.aim_fft_config(ctx, g.AIM_C128) == kernels
    for p, k in enumerate(kernels):
        assert ms[p, k] > 0 and ms[p, k] == ms[p, ms[p] > 0].min()
    # AUTO is never timed; the x-pass-only variants (small blocks, warp groups)
    # only on the x pass, the wide strided variant only on the others
    assert (ms[:, 0] == -1).all() and (ms[[0, 1, 3, 4]][:, [3, 4]] == -1).all() and ms[2, 5] == -1
    y = g.aim_matvec(ctx, xt, precision=g.AIM_C128).cpu().numpy()
    assert rel(y, op.matvec(x)) <= 1e-12
    g.aim_fft_config(ctx, g.AIM_C128, [g.AIM_FFT_AUTO] * 5)


def test_fft_config_rejects_bad_choices(plate_a):
    ctx, _ = plate_a
    with pytest.raises(g.AIMError):
        g.aim_fft_config(ctx, g.AIM_C64, [g.AIM_FFT_KERNELS, 0, 0, 0, 0])
    with pytest.raises(g.AIMError):
        g.aim_autotune(ctx, g.AIM_C64, nrhs=ctx.max_rhs + 1)
    assert g.aim_fft_config(ctx, g.AIM_C128) == [2, 2, 2, 2, 2]  # the built-in rule
    assert g.aim_fft_config(ctx, g.AIM_C64) == [2, 2, 2, 2, 2]


def test_stockham_fallback_length():
    """A padded length outside the four-step menu (18) runs the Stockham kernels."""
    v, t = plate_mesh(0.7, 6)
    ctx, op = make(v, t, max_rhs=2, planar=False)
    n, L, _ = g.aim_grid_info(ctx)
    assert L[0] == 18 and L[1] == 18 and L[2] == 5
    x = random_complex((2, ctx.N), 18)
    ref = op.matvec(x)
    for prec in WIDE:
        y = g.aim_matvec(ctx, torch.from_numpy(x).cuda(), precision=prec).cpu().numpy()
        assert rel(y, ref) <= 1e-12
    y32 = g.aim_matvec(ctx, torch.from_numpy(x.astype(np.complex64)).cuda()).cpu().numpy()
    assert rel(y32, ref) <= 1e-5


def test_all_pairs_near_equals_dense():
    """Near radius beyond the body: the product is the dense Galerkin matrix."""
    from oracle.efie import dense_Z

    v, t = plate_mesh(0.5, 4)
    ctx, op = make(v, t, radius=10.0)
    Z = dense_Z(op.rwg, K0)
    x = random_complex((1, ctx.N), 16)
    y = g.aim_matvec(ctx, torch.from_numpy(x).cuda()).cpu().numpy()
    assert rel(y[0], 0.5 * (Z + Z.T) @ x[0]) <= 1e-12


def test_ragged_grid_and_single_triangle_pair():
    # two triangles sharing one edge: N = 1, grid 3x3x3
    v = np.array([[0, 0, 0], [0.1, 0, 0.01], [0, 0.1, 0.02], [0.11, 0.1, 0.0]], dtype=np.float64)
    t = np.array([[0, 1, 2], [1, 3, 2]], dtype=np.int32)
    ctx, op = make(v, t)
    assert ctx.N == 1
    x = random_complex((1, 1), 17)
    y = g.aim_matvec(ctx, torch.from_numpy(x).cuda()).cpu().numpy()
    assert rel(y, op.matvec(x)) <= 1e-12


def test_invalid_inputs():
    v, t = plate_mesh(1.0, 2)
    with pytest.raises(g.AIMError):
        g.aim_setup(v, t, K0, -H)
    bad = t.copy()
    bad[0, 0] = 999
    with pytest.raises(g.AIMError):
        g.aim_setup(v, bad, K0, H)
    # a non-manifold edge: three triangles on one edge
    v3 = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1]], dtype=float) * 0.1
    t3 = np.array([[0, 1, 2], [0, 1, 3], [0, 1, 4]], dtype=np.int32)
    with pytest.raises(g.AIMError):
        g.aim_setup(v3, t3, K0, H)
    ctx = g.aim_setup(v, t, K0, H, max_rhs=1)
    x = torch.zeros((2, ctx.N), dtype=torch.complex128, device="cuda")
    with pytest.raises(g.AIMError):
        g.aim_matvec(ctx, x)  # nrhs > max_rhs


def test_zero_vector_gives_zero(plate_a):
    ctx, _ = plate_a
    x = torch.zeros((1, ctx.N), dtype=torch.complex128, device="cuda")
    assert torch.count_nonzero(g.aim_matvec(ctx, x)).item() == 0


@pytest.mark.slow
def test_full_size_sphere_sampled_rows():
    """4 lambda sphere (N = 58,080, grid 83^3 padded 180^3): sampled rows, both precisions."""
    R = 4.0
    v, t = icosphere_mesh(R, icosphere_frequency(R))
    rows = np.sort(np.random.default_rng(0).choice(30 * 44 * 44, 300, replace=False))
    ctx, op = make(v, t, near_rows=rows)
    assert ctx.N == 58080
    x = random_complex((1, ctx.N), 21)
    ref = op.matvec(x)[0, rows]
    for prec in WIDE:
        y = g.aim_matvec(ctx, torch.from_numpy(x).cuda(), precision=prec).cpu().numpy()[0, rows]
        assert rel(y, ref) <= 1e-12
    y32 = g.aim_matvec(ctx, torch.from_numpy(x.astype(np.complex64)).cuda()).cpu().numpy()[0, rows]
    assert rel(y32, ref) <= 1e-5


@pytest.mark.slow
def test_full_size_plate_32_lambda_multi_rhs_sampled_rows():
    """32 lambda plate (N = 248,256, grid 321x321x3 padded 648x648x5), 16 RHS (the
    lanes-over-RHS interpolation), sampled rows."""
    v, t = plate_mesh(32.0, 288)
    rows = np.sort(np.random.default_rng(1).choice(248256, 200, replace=False))
    ctx, op = make(v, t, max_rhs=16, near_rows=rows)
    assert ctx.N == 248256
    x = random_complex((16, ctx.N), 22)
    ref = op.matvec(x)[:, rows]
    y = g.aim_matvec(ctx, torch.from_numpy(x).cuda(), precision=g.AIM_C128).cpu().numpy()[:, rows]
    assert rel(y, ref) <= 1e-12
    y32 = g.aim_matvec(ctx, torch.from_numpy(x.astype(np.complex64)).cuda()).cpu().numpy()[:, rows]
    assert rel(y32, ref) <= 1e-5


def test_float_float_accuracy_beats_complex64_by_far(sphere_small):
    """The float-float product sits within a few 1e-14 of the native FP64 one."""
    ctx, op = sphere_small
    x = torch.from_numpy(random_complex((1, ctx.N), 23)).cuda()
    a = g.aim_matvec(ctx, x, precision=g.AIM_C128).cpu().numpy()
    b = g.aim_matvec(ctx, x, precision=g.AIM_C128_F64).cpu().numpy()
    assert rel(a, b) <= 1e-13


def test_planar_grid_collapses_to_one_plane(plate_a, plate_a_planar):
    """A plate on the z = 0 node plane: only that plane of the grid is kept, the
    convolution is two-dimensional, and the product is the oracle's (full 3-D
    grid) in every precision and batch size, including the lanes-over-RHS path."""
    ctx, op = plate_a_planar
    n, L, _ = g.aim_grid_info(ctx)
    assert n == [op.n[0], op.n[1], 1] and L == [op.L[0], op.L[1], 1]
    lam = g.aim_export(ctx, g.AIM_EXPORT_WEIGHTS)
    assert np.abs(lam - op.lam).max() <= 1e-12 * np.abs(op.lam).max()
    for nrhs, seed in ((1, 51), (3, 52), (17, 53)):
        x = random_complex((nrhs, ctx.N), seed)
        ref = op.matvec(x)
        for prec in WIDE:
            y = g.aim_matvec(ctx, torch.from_numpy(x).cuda(), precision=prec).cpu().numpy()
            assert rel(y, ref) <= 1e-12
        y32 = g.aim_matvec(ctx, torch.from_numpy(x.astype(np.complex64)).cuda()).cpu().numpy()
        assert rel(y32, op.matvec(x.astype(np.complex64).astype(np.complex128))) <= 1e-5
    # same product as the three-dimensional grid, to rounding
    ctx3, _ = plate_a
    x = torch.from_numpy(random_complex((3, ctx.N), 54)).cuda()
    a = g.aim_matvec(ctx, x, precision=g.AIM_C128_F64).cpu().numpy()
    b = g.aim_matvec(ctx3, x, precision=g.AIM_C128_F64).cpu().numpy()
    assert rel(a, b) <= 1e-13


def test_plate_off_node_plane_keeps_three_dimensions():
    """A plate between node planes has weights on every stencil plane: no collapse."""
    v, t = plate_mesh(1.0, 9)
    v = v.copy()
    v[:, 2] += 0.037
    ctx, op = make(v, t)
    n, L, _ = g.aim_grid_info(ctx)
    assert n == list(op.n) and n[2] == 3
    x = random_complex((1, ctx.N), 55)
    y = g.aim_matvec(ctx, torch.from_numpy(x).cuda()).cpu().numpy()
    assert rel(y, op.matvec(x)) <= 1e-12


@pytest.mark.slow
def test_full_size_sphere_16_lambda_sampled_rows():
    """16 lambda sphere (N = 908,280, grid 323^3 padded 648^3), the benchmark's
    workload: the complex64 product of 8 right-hand sides in the benchmark's
    launch configuration (FFT kernels autotuned), and with each FFT kernel
    forced on every pass (length-648 four-step pencils, the four-block
    strided kernel, the wide strided variant, the warp-group and small-block
    x passes, Stockham); then, on a one-RHS context, the FP64-accurate
    (float-float) and native FP64 products.  Sampled rows against the
    oracle's rows computed by direct summation of the grid convolution at
    their stencil nodes (its padded FFT would hold about 50 GB of host
    memory)."""
    R = 16.0
    v, t = icosphere_mesh(R, icosphere_frequency(R))
    rwg = RWG(v, t)
    assert rwg.N == 908280
    rows = np.sort(np.random.default_rng(7).choice(rwg.N, 32, replace=False))
    # inputs exactly representable in complex64, so one oracle evaluation serves every precision
    x = random_complex((8, rwg.N), 81).astype(np.complex64)
    op = oaim.AIMOperator(rwg, K0, H, 2, near_rows=rows)
    ref = op.matvec_rows(x.astype(np.complex128), rows)  # [8, 32]

    ctx = g.aim_setup(v, t, K0, H, M=2, near_radius=3 * H, max_rhs=8, precision=g.AIM_C64)
    n, L, _ = g.aim_grid_info(ctx)
    assert n == [323, 323, 323] and L == [648, 648, 648]
    xt = torch.from_numpy(x).cuda()
    for kernel in FFT_CHOICES:
        g.aim_fft_config(ctx, g.AIM_C64, [kernel] * 5)
        y = g.aim_matvec(ctx, xt, precision=g.AIM_C64).cpu().numpy()[:, rows]
        assert rel(y, ref) <= 1e-5, (kernel, rel(y, ref))
    g.aim_fft_config(ctx, g.AIM_C64, [g.AIM_FFT_AUTO] * 5)
    g.aim_autotune(ctx, g.AIM_C64, nrhs=8, reps=1)
    y = g.aim_matvec(ctx, xt, precision=g.AIM_C64).cpu().numpy()[:, rows]
    assert rel(y, ref) <= 1e-5
    ctx.close()
    del xt
    torch.cuda.empty_cache()

    ctx = g.aim_setup(v, t, K0, H, M=2, near_radius=3 * H, max_rhs=1, precision=g.AIM_C128)
    x1 = torch.from_numpy(x[:1].astype(np.complex128)).cuda()
    for prec in WIDE:
        y = g.aim_matvec(ctx, x1, precision=prec).cpu().numpy()[:, rows]
        assert rel(y, ref[:1]) <= 1e-12, (prec, rel(y, ref[:1]))
    ctx.close()


def test_mem_budget_and_non_finite_inputs():
    """opts.mem_budget: a context whose budget is exactly its footprint estimate
    (solver precision AIM_C128) runs FP64-accurate products, but a native-FP64
    product, whose grids the estimate does not count, is refused with
    AIM_ENOMEM and the context stays usable.  NaN or infinite plane-wave
    directions, right-hand sides and RCS angles are rejected with AIM_EINVAL."""
    from paper_1010_1456_gb300 import _lib

    v, t = plate_mesh(1.0, 9)
    est = g.aim_footprint(v, t, H, 2, 3 * H, 1, precision=g.AIM_C128)
    ctx, op = make(v, t)
    x = torch.from_numpy(random_complex((1, ctx.N), 91)).cuda()
    ref = op.matvec(x.cpu().numpy())
    ctx.close()
    ctx = g.aim_setup(v, t, K0, H, max_rhs=1, precision=g.AIM_C128, mem_budget=est)
    assert rel(g.aim_matvec(ctx, x, precision=g.AIM_C128).cpu().numpy(), ref) <= 1e-12
    with pytest.raises(g.AIMError) as e:
        g.aim_matvec(ctx, x, precision=g.AIM_C128_F64)
    assert e.value.code == _lib.AIM_ENOMEM
    assert rel(g.aim_matvec(ctx, x, precision=g.AIM_C128).cpu().numpy(), ref) <= 1e-12
    kh, po = planewave_minus_z_xpol()
    for bad in (np.nan, np.inf):
        kb = kh.copy()
        kb[0, 2] = bad
        with pytest.raises(g.AIMError) as e:
            g.aim_rhs_planewave(ctx, kb, po)
        assert e.value.code == _lib.AIM_EINVAL
    V = g.aim_rhs_planewave(ctx, kh, po)
    V[0, 5] = complex(np.nan, 0.0)
    with pytest.raises(g.AIMError) as e:
        g.aim_solve(ctx, V, 1e-6)
    assert e.value.code == _lib.AIM_EINVAL
    with pytest.raises(g.AIMError):
        g.aim_rcs(ctx, V, np.array([0.1, np.nan]), np.array([0.0, 0.0]))
    ctx.close()


@pytest.mark.parametrize("along", ["x", "y"])
def test_longest_padded_length_strip(along):
    """A 64 lambda x 1 lambda strip (576 x 9 lambda/9 squares) pads one axis to
    1296 = 36 x 36, the longest four-step length (the 64 lambda plate's):
    along x the fused x pass runs at 1296, along y the strided passes do; on
    the full three-dimensional grid (no plane collapse), every precision."""
    from aim_inputs import rect_plate_mesh

    v, t = rect_plate_mesh(64.0, 1.0, 576, 9) if along == "x" else rect_plate_mesh(1.0, 64.0, 9, 576)
    ctx, op = make(v, t, max_rhs=2, planar=False)
    n, L, _ = g.aim_grid_info(ctx)
    assert (L[0] if along == "x" else L[1]) == 1296
    x = random_complex((2, ctx.N), 95)
    ref = op.matvec(x)
    for prec in WIDE:
        y = g.aim_matvec(ctx, torch.from_numpy(x).cuda(), precision=prec).cpu().numpy()
        assert rel(y, ref) <= 1e-12, (prec, rel(y, ref))
    y32 = g.aim_matvec(ctx, torch.from_numpy(x.astype(np.complex64)).cuda()).cpu().numpy()
    assert rel(y32, op.matvec(x.astype(np.complex64).astype(np.complex128))) <= 1e-5
    ctx.close()
