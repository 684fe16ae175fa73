"""GB300-native AIM-accelerated EFIE method of moments.

Python binding of the C ABI in ``include/aim.h``: the functions below carry
the C names and only marshal arguments (torch tensors for device memory,
numpy arrays for host data).  Every step of the computation runs in the CUDA
library ``libaim.so``; if it is not built, the first call raises.

Complex vectors are torch tensors of shape [nrhs, N] (complex128 for AIM_C128,
complex64 for AIM_C64) on the current CUDA device.
"""

import ctypes as C

import numpy as np

from ._lib import (  # noqa: F401
    AIM_C64,
    AIM_C128,
    AIM_C128_F64,
    AIM_EXPORT_ANCHORS,
    AIM_EXPORT_DIAG,
    AIM_EXPORT_GHAT,
    AIM_EXPORT_MFIE_WEIGHTS,
    AIM_EXPORT_NEAR_COL,
    AIM_EXPORT_NEAR_PTR,
    AIM_EXPORT_NEAR_VAL,
    AIM_EXPORT_PROJ_PTR,
    AIM_EXPORT_WEIGHTS,
    AIM_ENOCONV,
    AIM_GMRES,
    AIM_TFQMR,
    AIMError,
    aim_mesh,
    aim_opts,
    aim_solve_info,
    check,
    load,
)

ETA0 = 376.730313668


def _torch():
    import torch

    return torch


class Context:
    """Owning handle of an ``aim_ctx*``; frees it on ``close()`` / garbage collection."""

    def __init__(self, handle, N, max_rhs, precision, M):
        self.handle = handle
        self.N = N
        self.max_rhs = max_rhs
        self.precision = precision
        self.M = M

    def close(self):
        if self.handle:
            load().aim_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def _mesh(verts, tris):
    v = np.ascontiguousarray(verts, dtype=np.float64)
    t = np.ascontiguousarray(tris, dtype=np.int32)
    m = aim_mesh(len(v), len(t), v.ctypes.data_as(C.POINTER(C.c_double)), t.ctypes.data_as(C.POINTER(C.c_int32)))
    return m, (v, t)


def _stream(stream):
    if stream is not None:
        return C.c_void_p(int(stream))
    torch = _torch()
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def aim_default_opts():
    o = aim_opts()
    load().aim_default_opts(C.byref(o))
    return o


def aim_setup(verts, tris, k, h, M=2, near_radius=None, precision=AIM_C128, restart=50, maxit=3000,
              check_every=5, max_rhs=1, stream=None, planar=True, verbose=False, cfie_alpha=1.0, mem_budget=0,
              krylov=AIM_GMRES):
    """Build a context (host FP64 setup + device spectrum); see aim_setup in aim.h."""
    lib = load()
    mesh, keep = _mesh(verts, tris)
    o = aim_default_opts()
    o.precision = precision
    o.restart = restart
    o.maxit = maxit
    o.check_every = check_every
    o.max_rhs = max_rhs
    o.stream = _stream(stream)
    o.planar = 1 if planar else 0
    o.verbose = 1 if verbose else 0
    o.cfie_alpha = float(cfie_alpha)
    o.mem_budget = int(mem_budget)
    o.krylov = int(krylov)
    h_ = C.c_void_p()
    r = 3.0 * h if near_radius is None else float(near_radius)
    check(lib.aim_setup(C.byref(mesh), float(k), float(h), int(M), r, C.byref(o), C.byref(h_)), "aim_setup")
    N = C.c_int64()
    check(lib.aim_num_unknowns(h_, C.byref(N)), "aim_num_unknowns")
    del keep
    return Context(h_, int(N.value), max_rhs, precision, M)


def aim_destroy(ctx):
    ctx.close()


def aim_set_stream(ctx, stream):
    """stream: a torch.cuda.Stream or a raw cudaStream_t handle (int)."""
    h = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    check(load().aim_set_stream(ctx.handle, C.c_void_p(h)), "aim_set_stream")


def aim_set_precision(ctx, precision):
    check(load().aim_set_precision(ctx.handle, int(precision)), "aim_set_precision")
    ctx.precision = precision


def aim_set_krylov(ctx, krylov):
    """AIM_GMRES or AIM_TFQMR for the context's next solves."""
    check(load().aim_set_krylov(ctx.handle, int(krylov)), "aim_set_krylov")


def aim_num_unknowns(ctx):
    N = C.c_int64()
    check(load().aim_num_unknowns(ctx.handle, C.byref(N)), "aim_num_unknowns")
    return int(N.value)


def aim_grid_info(ctx):
    n = (C.c_int32 * 3)()
    L = (C.c_int32 * 3)()
    nnz = C.c_int64()
    check(load().aim_grid_info(ctx.handle, n, L, C.byref(nnz)), "aim_grid_info")
    return list(n), list(L), int(nnz.value)


def _dev(t, dtype):
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != dtype or not t.is_contiguous():
        raise ValueError(f"expected a contiguous CUDA tensor of dtype {dtype}")
    return C.c_void_p(t.data_ptr())


def aim_rhs_planewave(ctx, khat, pol, V=None):
    """V[nrhs, N] (complex128, device) for plane waves exp(-j k khat.r) pol."""
    torch = _torch()
    kh = np.ascontiguousarray(np.atleast_2d(khat), dtype=np.float64)
    po = np.ascontiguousarray(np.atleast_2d(pol), dtype=np.float64)
    nrhs = len(kh)
    if V is None:
        V = torch.empty((nrhs, ctx.N), dtype=torch.complex128, device="cuda")
    check(load().aim_rhs_planewave(ctx.handle, nrhs, kh.ctypes.data_as(C.POINTER(C.c_double)),
                                   po.ctypes.data_as(C.POINTER(C.c_double)), _dev(V, torch.complex128)),
          "aim_rhs_planewave")
    return V


def aim_matvec(ctx, x, y=None, precision=None):
    """y = Z~ x on the device (enqueued on the context stream)."""
    torch = _torch()
    if precision is None:
        precision = AIM_C128 if x.dtype == torch.complex128 else AIM_C64
    dt = torch.complex64 if precision == AIM_C64 else torch.complex128
    x2 = x.reshape(-1, ctx.N)
    if y is None:
        y = torch.empty_like(x2)
    check(load().aim_matvec(ctx.handle, _dev(x2, dt), _dev(y, dt), x2.shape[0], precision), "aim_matvec")
    return y


def aim_matvec_host(ctx, x, precision=AIM_C128, out=None):
    """Same product with host buffers, copies included; synchronises.

    x: numpy array, or a CPU torch tensor (pinned memory copies fastest);
    out: optional host buffer of the same kind and shape for the result."""
    if hasattr(x, "data_ptr"):  # torch tensor in host memory
        torch = _torch()
        dt = torch.complex64 if precision == AIM_C64 else torch.complex128
        if x.device.type != "cpu" or x.dtype != dt or not x.is_contiguous():
            raise ValueError(f"x: contiguous host tensor of {dt} expected")
        x2 = x.reshape(-1, ctx.N)
        y = torch.empty_like(x2) if out is None else out
        if y.shape != x2.shape or y.dtype != dt or y.device.type != "cpu" or not y.is_contiguous():
            raise ValueError("out: contiguous host tensor shaped like x expected")
        check(load().aim_matvec_host(ctx.handle, C.c_void_p(x2.data_ptr()), C.c_void_p(y.data_ptr()), x2.shape[0],
                                     precision), "aim_matvec_host")
        return y
    dt = np.complex64 if precision == AIM_C64 else np.complex128
    x = np.ascontiguousarray(np.atleast_2d(x), dtype=dt)
    y = np.empty_like(x) if out is None else out
    check(load().aim_matvec_host(ctx.handle, x.ctypes.data_as(C.c_void_p), y.ctypes.data_as(C.c_void_p),
                                 x.shape[0], precision), "aim_matvec_host")
    return y


def aim_solve(ctx, V, tol=1e-6, X=None, raise_on_noconv=True):
    """Solve Z~ X = V (device complex128 [nrhs, N]); returns (X, info dict)."""
    torch = _torch()
    V2 = V.reshape(-1, ctx.N)
    nrhs = V2.shape[0]
    if X is None:
        X = torch.empty_like(V2)
    rel = (C.c_double * nrhs)()
    conv = (C.c_int32 * nrhs)()
    info = aim_solve_info(0, 0, C.cast(rel, C.POINTER(C.c_double)), C.cast(conv, C.POINTER(C.c_int32)))
    code = load().aim_solve(ctx.handle, _dev(V2, torch.complex128), _dev(X, torch.complex128), nrhs, float(tol),
                            C.byref(info))
    if code != 0 and not (code == AIM_ENOCONV and not raise_on_noconv):
        check(code, "aim_solve")
    return X, {
        "iterations": info.iterations,
        "restarts": info.restarts,
        "rel_res": np.array(rel[:]),
        "converged": np.array(conv[:], dtype=bool),
        "status": code,
    }


class Pack:
    """Owning handle of an ``aim_pack*`` (aim_pack_create): several contexts
    batched through one launch per product stage.  ``ld`` is the packed row
    length, ``B`` the total of right-hand sides, ``b0[i]`` the first row of
    instance i.  The contexts must outlive the pack."""

    def __init__(self, handle, ctxs, nrhs, ld, B, b0):
        self.handle = handle
        self.ctxs = list(ctxs)
        self.nrhs = list(nrhs)
        self.ld = ld
        self.B = B
        self.b0 = b0

    def close(self):
        if self.handle:
            load().aim_pack_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def rows(self, i):
        """(first row, end row, columns) of instance i in the packed vectors."""
        return self.b0[i], self.b0[i] + self.nrhs[i], self.ctxs[i].N

    def pack(self, parts, dtype=None):
        """Packed [B, ld] device tensor (zero padding) from per-instance [nrhs_i, N_i] tensors."""
        torch = _torch()
        dtype = parts[0].dtype if dtype is None else dtype
        out = torch.zeros((self.B, self.ld), dtype=dtype, device=parts[0].device)
        for i, p in enumerate(parts):
            r0, r1, n = self.rows(i)
            out[r0:r1, :n] = p.reshape(r1 - r0, n)
        return out

    def unpack(self, X):
        """Per-instance [nrhs_i, N_i] views of a packed tensor."""
        out = []
        for i in range(len(self.ctxs)):
            r0, r1, n = self.rows(i)
            out.append(X[r0:r1, :n])
        return out


def aim_pack_create(ctxs, nrhs):
    """Pack contexts (sharing device, k, h, M and stencil layout) with nrhs[i]
    right-hand sides each; see aim_pack_create in aim.h."""
    lib = load()
    K = len(ctxs)
    hs = (C.c_void_p * K)(*[c.handle for c in ctxs])
    nr = (C.c_int32 * K)(*[int(n) for n in nrhs])
    h_ = C.c_void_p()
    check(lib.aim_pack_create(hs, K, nr, C.byref(h_)), "aim_pack_create")
    ld = C.c_int64()
    B = C.c_int32()
    b0 = (C.c_int32 * K)()
    check(lib.aim_pack_dims(h_, C.byref(ld), C.byref(B), b0), "aim_pack_dims")
    return Pack(h_, ctxs, nrhs, int(ld.value), int(B.value), [int(v) for v in b0])


def aim_pack_set_stream(pack, stream):
    h = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    check(load().aim_pack_set_stream(pack.handle, C.c_void_p(h)), "aim_pack_set_stream")


def aim_pack_matvec(pack, x, y=None, precision=None):
    """y = Z~ x on packed [B, ld] vectors (complex64: one launch per stage)."""
    torch = _torch()
    if precision is None:
        precision = AIM_C128 if x.dtype == torch.complex128 else AIM_C64
    dt = torch.complex64 if precision == AIM_C64 else torch.complex128
    if y is None:
        y = torch.empty_like(x)
    check(load().aim_pack_matvec(pack.handle, _dev(x, dt), _dev(y, dt), int(precision)), "aim_pack_matvec")
    return y


def aim_pack_solve(pack, V, tol=1e-6, X=None, raise_on_noconv=True):
    """Solve every instance's system at once (packed complex128 [B, ld]); returns (X, info dict)."""
    torch = _torch()
    if X is None:
        X = torch.empty_like(V)
    B = pack.B
    rel = (C.c_double * B)()
    conv = (C.c_int32 * B)()
    info = aim_solve_info(0, 0, C.cast(rel, C.POINTER(C.c_double)), C.cast(conv, C.POINTER(C.c_int32)))
    code = load().aim_pack_solve(pack.handle, _dev(V, torch.complex128), _dev(X, torch.complex128), float(tol),
                                 C.byref(info))
    if code != 0 and not (code == AIM_ENOCONV and not raise_on_noconv):
        check(code, "aim_pack_solve")
    return X, {
        "iterations": info.iterations,
        "restarts": info.restarts,
        "rel_res": np.array(rel[:]),
        "converged": np.array(conv[:], dtype=bool),
        "status": code,
    }


def aim_rcs(ctx, X, theta, phi):
    """(sigma_thth, sigma_phph) [nrhs, ndir] (numpy) of device currents X."""
    torch = _torch()
    X2 = X.reshape(-1, ctx.N)
    th = np.ascontiguousarray(theta, dtype=np.float64).ravel()
    ph = np.ascontiguousarray(phi, dtype=np.float64).ravel()
    nrhs, nd = X2.shape[0], len(th)
    stt = np.empty((nrhs, nd))
    spp = np.empty((nrhs, nd))
    dp = C.POINTER(C.c_double)
    check(load().aim_rcs(ctx.handle, _dev(X2, torch.complex128), nrhs, nd, th.ctypes.data_as(dp),
                         ph.ctypes.data_as(dp), stt.ctypes.data_as(dp), spp.ctypes.data_as(dp)), "aim_rcs")
    return stt, spp


def aim_footprint(verts, tris, h, M=2, near_radius=None, max_rhs=1, cfie_alpha=1.0, precision=AIM_C128):
    """Estimated device bytes of a context that has solved with solver precision ``precision``."""
    mesh, keep = _mesh(verts, tris)
    b = C.c_size_t()
    r = 3.0 * h if near_radius is None else float(near_radius)
    check(load().aim_footprint(C.byref(mesh), float(h), int(M), r, int(max_rhs), float(cfie_alpha), int(precision),
                               C.byref(b)), "aim_footprint")
    return int(b.value)


def aim_export(ctx, what):
    """Copy an internal setup array to host numpy (see AIM_EXPORT_* in aim.h)."""
    n, L, nnz = aim_grid_info(ctx)
    N = ctx.N
    S = (ctx.M + 1) ** 3
    shapes = {
        AIM_EXPORT_ANCHORS: ((N, 3), np.int32),
        AIM_EXPORT_WEIGHTS: ((N, 4, S), np.float64),
        AIM_EXPORT_NEAR_PTR: ((N + 1,), np.int32),
        AIM_EXPORT_NEAR_COL: ((nnz,), np.int32),
        AIM_EXPORT_NEAR_VAL: ((nnz,), np.complex128),
        AIM_EXPORT_DIAG: ((N,), np.complex128),
        AIM_EXPORT_GHAT: ((L[2] // 2 + 1, L[1] // 2 + 1, L[0] // 2 + 1), np.complex128),
        AIM_EXPORT_PROJ_PTR: ((n[0] * n[1] * n[2] + 1,), np.int32),
        AIM_EXPORT_MFIE_WEIGHTS: ((N, 3, S), np.float64),
    }
    shape, dt = shapes[what]
    a = np.empty(shape, dtype=dt)
    check(load().aim_export(ctx.handle, what, a.ctypes.data_as(C.c_void_p), a.nbytes), "aim_export")
    return a


def aim_launch_count(ctx):
    c = C.c_int64()
    check(load().aim_launch_count(ctx.handle, C.byref(c)), "aim_launch_count")
    return int(c.value)


def aim_profile(ctx, mode):
    """1: time every kernel launch with CUDA events; 0: stop; 2: clear totals."""
    check(load().aim_profile(ctx.handle, int(mode)), "aim_profile")


def aim_profile_read(ctx, max_kernels=64):
    """{kernel name: (launches, total ms)} since profiling started (synchronises)."""
    names = C.create_string_buffer(48 * max_kernels)
    launches = (C.c_int64 * max_kernels)()
    ms = (C.c_double * max_kernels)()
    cnt = C.c_int()
    check(load().aim_profile_read(ctx.handle, max_kernels, names, launches, ms, C.byref(cnt)), "aim_profile_read")
    out = {}
    for i in range(min(cnt.value, max_kernels)):
        nm = names.raw[48 * i : 48 * (i + 1)].split(b"\0", 1)[0].decode()
        out[nm] = (int(launches[i]), float(ms[i]))
    return out


def aim_probe_fma_peak(which=64):
    t = C.c_double()
    check(load().aim_probe_fma_peak(int(which), C.byref(t)), "aim_probe_fma_peak")
    return float(t.value)


(AIM_FFT_AUTO, AIM_FFT_STOCKHAM, AIM_FFT_FOURSTEP, AIM_FFT_FOURSTEP_SMALL, AIM_FFT_FOURSTEP_WARP,
 AIM_FFT_FOURSTEP_WIDE) = range(6)
AIM_FFT_KERNELS = 6
FFT_PASSES = ("fft_z_fwd", "fft_y_fwd", "fft_x_conv", "fft_y_inv", "fft_z_inv")


def aim_fft_config(ctx, precision=AIM_C128, kernels=None):
    """Set (kernels: five AIM_FFT_* values, or None) and return the FFT kernel of each pass."""
    lib = load()
    get = (C.c_int32 * 5)()
    st = None
    if kernels is not None:
        if len(kernels) != 5:
            raise ValueError("kernels: one AIM_FFT_* value per pass (5)")
        st = (C.c_int32 * 5)(*[int(k) for k in kernels])
    check(lib.aim_fft_config(ctx.handle, int(precision), st, get), "aim_fft_config")
    return [int(k) for k in get]


def aim_autotune(ctx, precision=AIM_C128, nrhs=1, reps=3):
    """Time each FFT kernel per pass, keep the fastest.  Returns (kernels, ms[5][AIM_FFT_KERNELS])."""
    lib = load()
    k = (C.c_int32 * 5)()
    ms = (C.c_double * (5 * AIM_FFT_KERNELS))()
    check(lib.aim_autotune(ctx.handle, int(precision), int(nrhs), int(reps), k, ms), "aim_autotune")
    return [int(v) for v in k], np.array(list(ms)).reshape(5, AIM_FFT_KERNELS)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def rcs_direction_grid(n_theta, n_phi=None):
    """(theta, phi, weight) of the eq. (1) quadrature (aim_rcs_grid): Gauss-Legendre
    in cos(theta) times uniform phi, flattened theta-major."""
    n_phi = 2 * n_theta if n_phi is None else n_phi
    nd = int(n_theta) * int(n_phi)
    th, ph, w = np.empty(nd), np.empty(nd), np.empty(nd)
    dp = C.POINTER(C.c_double)
    check(load().aim_rcs_grid(int(n_theta), int(n_phi), th.ctypes.data_as(dp), ph.ctypes.data_as(dp),
                              w.ctypes.data_as(dp)), "aim_rcs_grid")
    return th, ph, w


def err_thth(sigma, sigma_ref, weight):
    """Eq. (1) (aim_err_thth): relative RMS difference of bistatic RCS patterns
    [nrhs, ndir] (or [ndir]) against a reference of the same shape."""
    s = _f64(np.atleast_2d(sigma))
    r = _f64(np.broadcast_to(np.atleast_2d(sigma_ref), s.shape))
    w = _f64(weight)
    out = np.empty(s.shape[0])
    dp = C.POINTER(C.c_double)
    check(load().aim_err_thth(s.shape[0], s.shape[1], s.ctypes.data_as(dp), r.ctypes.data_as(dp),
                              w.ctypes.data_as(dp), out.ctypes.data_as(dp)), "aim_err_thth")
    return out if np.ndim(sigma) > 1 else out[0]


def mie_sigma_thth(radius, theta, phi, k=2.0 * np.pi):
    """Mie-series sigma_thth of a PEC sphere lit by an x-polarised wave travelling -z
    (aim_mie_sigma_thth), at directions theta, phi (flattened)."""
    th, ph = _f64(np.ravel(theta)), _f64(np.ravel(phi))
    out = np.empty(len(th))
    dp = C.POINTER(C.c_double)
    check(load().aim_mie_sigma_thth(float(radius), float(k), len(th), th.ctypes.data_as(dp), ph.ctypes.data_as(dp),
                                    out.ctypes.data_as(dp)), "aim_mie_sigma_thth")
    return out
