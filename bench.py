#!/usr/bin/env python3
"""Benchmark of the AIM matrix-vector product and solve on synthetic PEC scatterers.

Default workload: the 16 lambda PEC sphere of the paper's sphere family
(Section 2.1, Table 2; geodesic icosphere at mean edge <= lambda/9,
N = 908,280 RWG unknowns, grid 323^3 zero-padded to 648^3, h = lambda/10,
27-point stencils, near radius 3h) with 8 right-hand sides: the largest
configuration that fits one GPU.  A step is one complex64 AIM product of the
8 vectors (projection, five FFT passes, interpolation and near correction)
through the C ABI; the inputs are resident in HBM, the product's working set
(~60 GB of grids) exceeds L2 and L2 is also flushed between steps.  Beside
the product the line reports the plain single-RHS FP64 products, the mixed
(complex64 Arnoldi, FP64-accurate refinement) and plain FP64-accurate CFIE
solves (alpha = 0.6) of the paper's excitation with err_thth (eq. 1) of
both against the Mie series, a short serving stream (p50/p99), the
end-to-end rate through host buffers and the oracle timed on the host.

  python bench.py [--gpus N --steps K --warmup W] [--workload NAME] [--impl ours|reference]

One JSON line on stdout (rank 0).  Multi-GPU runs are replicas: each rank
solves its own copy (no data-path collective), value = total products / time.
"""

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "AIM matvec/s and served solves/s (p50/p99) at stated err, vs FP64 plain path"
ETA0 = 376.730313668
K0 = 2.0 * np.pi
H = 0.1

WORKLOADS = {
    # name: (kind, size, nrhs, precision); "c128" = FP64-accurate product with
    # float-float FFT passes, "f64" = native FP64 throughout, "c64" = complex64
    "pec-sphere-r4lambda-fp64-1rhs": ("sphere", 4.0, 1, "c128"),
    "pec-sphere-r4lambda-nativefp64-1rhs": ("sphere", 4.0, 1, "f64"),
    "pec-sphere-r4lambda-c64-1rhs": ("sphere", 4.0, 1, "c64"),
    "pec-plate-1lambda-fp64-1rhs": ("plate", 1.0, 1, "c128"),
    "pec-plate-32lambda-c64-64rhs": ("plate", 32.0, 64, "c64"),
    "pec-sphere-r16lambda-c64-8rhs": ("sphere", 16.0, 8, "c64"),
}
PRECISION = {"c128": 2, "f64": 3, "c64": 1}  # AIM_C128, AIM_C128_F64, AIM_C64
DEFAULT = "pec-sphere-r16lambda-c64-8rhs"


def mesh_for(kind, size):
    from aim_inputs import icosphere_frequency, icosphere_mesh, plate_mesh

    if kind == "plate":
        return plate_mesh(size, int(round(9 * size)))
    return icosphere_mesh(size, icosphere_frequency(size))


# ---------------------------------------------------------------- kernel models
def kernel_models(N, n, L, nnz, nent, S, nrhs, e, touched=None, projected=None):
    """Algorithmic bytes and flops per launch of each product kernel.

    e = bytes per complex value, w = bytes per real weight.  FFT flops use
    the 5 L log2 L convention per length-L transform.  touched = grid nodes
    that lie in some stencil (the interpolation reads only those); projected
    = grid nodes the projection writes (the nodes of its 8-node groups with
    entries when the grid keeps the zeros of the others, else every node);
    both default to all nodes.
    """
    nx, ny, nz = n
    Lx, Ly, Lz = L
    G = 4 * nrhs
    w = e // 2
    Nc = nx * ny * nz
    lg = np.log2
    oct_ = (Lx // 2 + 1) * (Ly // 2 + 1) * (Lz // 2 + 1)
    m = {}
    npj = Nc if projected is None else projected
    m["proj_gather"] = (nent * (4 + 4 * w) + (npj + 1) * 4 + nrhs * N * e + G * npj * e, 16.0 * nent * nrhs)
    m["fft_z_fwd"] = (G * (Nc + Lz * ny * nx) * e, G * nx * ny * 5.0 * Lz * lg(Lz))
    m["fft_y_fwd"] = (G * (Lz * ny * nx + Lz * Ly * nx) * e, G * nx * Lz * 5.0 * Ly * lg(Ly))
    m["fft_x_conv"] = (2 * G * Lz * Ly * nx * e + oct_ * e, G * Ly * Lz * (10.0 * Lx * lg(Lx) + 6.0 * Lx))
    m["fft_y_inv"] = m["fft_y_fwd"]
    m["fft_z_inv"] = m["fft_z_fwd"]
    m["transpose_phi"] = (2.0 * G * Nc * e, 0.0)
    m["transpose_x"] = (2.0 * nrhs * N * e, 0.0)
    m["x_to_ff"] = (2.0 * nrhs * N * 16, 0.0)
    nt = Nc if touched is None else touched
    m["interp_near"] = (
        G * nt * e + N * 4 * S * w + N * 4 + nnz * (e + 4) + (N + 1) * 4 + 2 * nrhs * N * e,
        nrhs * (16.0 * N * S + 8.0 * nnz),
    )
    return m


FFT_SOURCES = ("fft.cu", "common.h", "ff.h", "fft_policy.h", "fft4.cuh", "fft4_launch.cuh", "fft4_p32.cu",
               "fft4_p64.cu", "fft4_pff.cu")
KERNEL_SOURCES = {
    "proj_gather": ("matvec.cu", "common.h", "ff.h"),
    "interp_near": ("matvec.cu", "common.h", "ff.h"),
}


# FP32 flops per complex float-float operation, from csrc/ff.h and the PFF
# policy in csrc/fft.cu: lazy add = TwoSum (6) + 2 adds; product by a real
# constant = 2 x (mul + 3 FMA + FastTwoSum) = 2 x 10; complex product =
# 2 x ff_dot2 (2 mul + TwoSum + 6 FMA + 2 add + FastTwoSum = 26).  FMA = 2 flops.
FF_CADD, FF_CMULR, FF_CMUL = 16, 20, 52


def ff_transform_flops(L, pruned_first=False):
    """FP32 flops of one length-L float-float Stockham transform (radices 4, 3, 5, 2)."""
    rad = []
    x = L
    for r in (4, 3, 5, 2):
        while x % r == 0:
            rad.append(r)
            x //= r
    per_bfly = {2: 2 * FF_CADD, 3: 6 * FF_CADD + FF_CMULR, 4: 8 * FF_CADD, 5: 16 * FF_CADD + 8 * FF_CMULR}
    total, Ns = 0.0, 1
    for s, r in enumerate(rad):
        nb = L // r
        bf = per_bfly[r]
        if s == 0 and r == 4 and pruned_first:
            bf = 4 * FF_CADD
        if Ns > 1:
            bf += (r - 1) * FF_CMUL  # twiddles
        total += nb * bf
        Ns *= r
    return total


def ff_fft_flops(kernel, n, L, nrhs):
    """FP32 flops per launch of a float-float FFT pass (first forward stage pruned when n <= L/2)."""
    nx, ny, nz = n
    Lx, Ly, Lz = L
    G = 4 * nrhs
    if kernel == "fft_x_conv":
        return G * Ly * Lz * (ff_transform_flops(Lx, 2 * nx <= Lx) + ff_transform_flops(Lx) + Lx * FF_CMUL)
    if kernel in ("fft_y_fwd", "fft_y_inv"):
        return G * nx * Lz * ff_transform_flops(Ly, kernel == "fft_y_fwd" and 2 * ny <= Ly)
    if kernel in ("fft_z_fwd", "fft_z_inv"):
        return G * nx * ny * ff_transform_flops(Lz, kernel == "fft_z_fwd" and 2 * nz <= Lz)
    return None


def source_digest(kernel):
    """Hash of the source files a kernel is built from (FFT_SOURCES for the FFT passes)."""
    files = KERNEL_SOURCES.get(kernel, FFT_SOURCES)
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1010_1456_gb300", "csrc")
    for f in files:
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:12]


def ncu_traffic(workload, kernel):
    """DRAM bytes per launch from the committed ncu summary, if the sources still match."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    if not os.path.exists(path):
        return None
    dig = source_digest(kernel)
    for line in open(path):
        p = line.split()
        if len(p) == 4 and p[0] == workload and p[1] == kernel and p[2] == dig:
            return float(p[3])
    return None


def aggregate(total_ms, steps, nrhs, world, device=None):
    """Whole-job rate of independent replicas: every rank timed `steps` products
    of `nrhs` vectors; the job time is the slowest rank's (max over ranks)."""
    if world > 1:
        import torch

        t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
    return total_ms, world * steps * nrhs / (total_ms * 1e-3)


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            t0 = time.perf_counter()
            while not self.rows and time.perf_counter() - t0 < 5.0:  # sampler is live before timing starts
                time.sleep(0.02)
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                for nm, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- oracle timing
class OracleSample:
    """The oracle's AIM product, as it stands, timed on this host in bounded pieces.

    The oracle's near-zone setup for all rows of a large problem takes far
    longer than a bench run, so its near matrix is built for a seeded sample
    of rows.  One timed piece is a quarter of one right-hand side's product:
    the projection, padded FFT convolution and interpolation of one grid
    component (x, y, z current or charge, in turn), plus a quarter of the
    near SpMV (the sampled rows' time scaled by N / rows).  Four pieces make
    one product, so products/s = 0.25 x pieces / time.
    """

    def __init__(self, verts, tris, sample_rows=192, seed=0):
        from oracle import aim as oaim
        from oracle.rwg import RWG

        t0 = time.perf_counter()
        rwg = RWG(verts, tris)
        rng = np.random.default_rng(seed)
        self.rows = np.sort(rng.choice(rwg.N, min(sample_rows, rwg.N), replace=False))
        self.op = oaim.AIMOperator(rwg, K0, H, 2, near_rows=self.rows)
        _ = self.op.Ghat  # the padded spectrum, built once outside the timed pieces
        self.N = rwg.N
        self.setup_s = time.perf_counter() - t0
        self.t = []
        self.comp = 0

    def piece(self, x):
        """Time one quarter product of x [1, N]; returns its seconds."""
        op, c = self.op, self.comp
        self.comp = (self.comp + 1) % 4
        t0 = time.perf_counter()
        op.interpolate(op.convolve(op.project(x, comps=[c])), comps=[c])
        t1 = time.perf_counter()
        op.Znear @ x[0]
        t2 = time.perf_counter()
        dt = (t1 - t0) + 0.25 * (t2 - t1) * (self.N / len(self.rows))
        self.t.append(dt)
        return dt

    def result(self, warm=0):
        t = self.t[warm:]
        return {
            "value": 0.25 * len(t) / sum(t),
            "unit": "matvec/s",
            "cores": os.cpu_count(),
            "kind": "oracle",
            "sample": f"{len(t)} timed quarter products of one RHS (NumPy/SciPy FP64, scipy.fft workers="
                      f"{os.cpu_count()}): projection, padded FFT convolution and interpolation of one grid "
                      f"component in turn, plus a quarter of the near SpMV timed on {len(self.rows)} seeded rows "
                      f"and scaled by N/{len(self.rows)}; 4 pieces = 1 product; oracle setup "
                      f"{self.setup_s:.0f} s outside the timing",
        }


def oracle_matvec_rate(verts, tris, budget_s=20.0, seed=0):
    """cpu_baseline: the oracle sample timed for about budget_s seconds (one warm-up piece)."""
    from aim_inputs import random_complex

    o = OracleSample(verts, tris, seed=seed)
    x = random_complex((1, o.N), seed + 1)
    o.piece(x)
    t_start = time.perf_counter()
    while len(o.t) < 2 or (time.perf_counter() - t_start < budget_s and len(o.t) < 200):
        o.piece(x)
    return o.result(warm=1)


# ---------------------------------------------------------------- solves
def solve_section(g, ctx, kind, size, nrhs, P0):
    """EFIE solves of an open scatterer (plate): plain native FP64, FP64-accurate
    and mixed (complex64 + FP64 refinement), tol 1e-6; err_thth of the mixed
    and FP64-accurate RCS against the plain RCS by eq. (1)."""
    import torch

    from aim_inputs import planewave_minus_z_xpol, random_incidence

    if nrhs == 1:
        kh, po = planewave_minus_z_xpol()
    else:
        kh, po = random_incidence((nrhs + 1) // 2, seed=0)
        kh, po = kh[:nrhs], po[:nrhs]
    V = g.aim_rhs_planewave(ctx, kh, po)
    ka = K0 * (size if kind == "sphere" else size / np.sqrt(2.0))
    nth = max(64, 4 * int(np.ceil(ka)))
    th, ph, w = g.rcs_direction_grid(nth)
    out = {}
    sig = {}
    runs = (("plain_fp64", g.AIM_C128_F64), ("fp64_float_float_fft", g.AIM_C128), ("mixed_c64_fp64_refined", g.AIM_C64))
    if ctx.N * nrhs > 4_000_000:
        # batches this large would keep the FP64 solves running for many minutes:
        # only the mixed solve, its RCS compared with nothing
        out["skipped"] = "plain_fp64 and fp64_float_float_fft: N x nrhs > 4e6"
        runs = runs[2:]
    for name, P in runs:
        g.aim_set_precision(ctx, P)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        X, info = g.aim_solve(ctx, V, 1e-6, raise_on_noconv=False)
        t = time.perf_counter() - t0
        sig[name] = g.aim_rcs(ctx, X, th, ph)[0]
        out[name] = {"time_s": t, "solves_per_s": 1.0 / t, "rhs_per_s": nrhs / t, "iterations": info["iterations"],
                     "restarts": info["restarts"], "max_rel_res": float(info["rel_res"].max()),
                     "converged": bool(info["converged"].all())}
    # where the mixed solve's time goes: device time per kernel (a second,
    # profiled run) against its wall time
    g.aim_set_precision(ctx, g.AIM_C64)
    g.aim_profile(ctx, 2)
    g.aim_profile(ctx, 1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g.aim_solve(ctx, V, 1e-6, raise_on_noconv=False)
    wall = time.perf_counter() - t0
    g.aim_profile(ctx, 0)
    prof = g.aim_profile_read(ctx)
    g.aim_profile(ctx, 2)
    dev = sum(ms for _, ms in prof.values())
    top = sorted(prof.items(), key=lambda kv: -kv[1][1])[:12]
    out["mixed_profile"] = {"wall_s_profiled": wall, "device_s": dev / 1e3,
                            "launches": int(sum(c for c, _ in prof.values())),
                            "top": {k: {"launches": c, "ms": round(ms, 3)} for k, (c, ms) in top}}
    g.aim_set_precision(ctx, P0)
    if "plain_fp64" in sig:
        out["err_thth_mixed_vs_plain"] = float(np.max(g.err_thth(sig["mixed_c64_fp64_refined"], sig["plain_fp64"], w)))
        out["err_thth_float_float_vs_plain"] = float(np.max(g.err_thth(sig["fp64_float_float_fft"], sig["plain_fp64"],
                                                                       w)))
        out["speedup_mixed_over_plain"] = out["plain_fp64"]["time_s"] / out["mixed_c64_fp64_refined"]["time_s"]
    out["rcs_directions"] = int(len(th))
    return out


SOLVE_RESTART = 120


def solve_section_sphere(g, verts, tris, radius, nrhs, stream):
    """CFIE (alpha = 0.6, the paper's formulation for closed bodies, Section 2.2)
    solves of the sphere, tol 1e-6 on the true residual:

    * mixed: the whole batch in one solve, complex64 Arnoldi products with
      FP64-accurate (float-float) true residuals at every restart;
    * plain: the -z pair (x and y polarisation) one right-hand side at a
      time, every product FP64-accurate (the plain single-RHS FP64 path).

    Right-hand sides: 8 or more -> the four travel directions -z, -x, -y,
    -(1,1,1)/sqrt3 with theta/phi polarisation (the first two are the -z
    pair, x and y polarised); 1 -> the x-polarised wave travelling -z.
    err_thth (eq. 1) of both against the Mie series on the -z pair; first
    solves (one-time allocations and graph capture included)."""
    import torch

    from aim_inputs import planewave_minus_z_xpol, sphere_four_directions

    if nrhs >= 8:
        kh, po = sphere_four_directions()
        kh, po = kh[:nrhs], po[:nrhs]
        nrhs = len(kh)
    else:
        kh, po = planewave_minus_z_xpol(1)
        nrhs = 1
    npair = min(2, nrhs)
    t0 = time.perf_counter()
    # GMRES(120): the sphere's Arnoldi process fits one cycle, so the mixed solve pays one FP64-accurate
    # residual product of the batch per cycle less often (both arms use the same context)
    ctx = g.aim_setup(verts, tris, K0, H, M=2, near_radius=3 * H, max_rhs=nrhs, precision=g.AIM_C64,
                      stream=stream.cuda_stream, cfie_alpha=0.6, restart=SOLVE_RESTART)
    setup_s = time.perf_counter() - t0
    V = g.aim_rhs_planewave(ctx, kh, po)
    out = {"formulation": "CFIE alpha = 0.6", "setup_s": setup_s, "nrhs_mixed": nrhs, "tol": 1e-6,
           "krylov": f"GMRES({SOLVE_RESTART}), diagonal preconditioner",
           "rhs": "four directions -z, -x, -y, -(1,1,1)/sqrt3 x (theta, phi) polarisation" if nrhs >= 8
           else "x-polarised wave travelling -z"}
    # mixed: the whole batch
    g.aim_set_precision(ctx, g.AIM_C64)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    Xm, info = g.aim_solve(ctx, V, 1e-6, raise_on_noconv=False)
    tm = time.perf_counter() - t0
    out["mixed_c64_fp64_refined"] = {"time_s": tm, "solves_per_s": nrhs / tm, "iterations": info["iterations"],
                                     "restarts": info["restarts"], "max_rel_res": float(info["rel_res"].max()),
                                     "converged": bool(info["converged"].all())}
    # plain: one right-hand side at a time, FP64-accurate products
    g.aim_set_precision(ctx, g.AIM_C128)
    Xp = torch.empty((npair, ctx.N), dtype=torch.complex128, device=V.device)
    tp, its, res, conv = 0.0, [], [], []
    for b in range(npair):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Xb, ib = g.aim_solve(ctx, V[b : b + 1].contiguous(), 1e-6, raise_on_noconv=False)
        tp += time.perf_counter() - t0
        Xp[b] = Xb[0]
        its.append(ib["iterations"])
        res.append(float(ib["rel_res"].max()))
        conv.append(bool(ib["converged"].all()))
    out["plain_fp64_accurate_single_rhs"] = {"time_s": tp, "solves": npair, "solves_per_s": npair / tp,
                                             "iterations": its, "max_rel_res": max(res), "converged": all(conv)}
    out["speedup_mixed_over_plain_solves_per_s"] = (nrhs / tm) / (npair / tp)
    # RCS and eq. (1) against the Mie series on the -z pair
    ka = K0 * radius
    nth = max(64, 4 * int(np.ceil(ka)))
    th, ph, w = g.rcs_direction_grid(nth)
    t0 = time.perf_counter()
    sm = g.aim_rcs(ctx, Xm[:npair].contiguous(), th, ph)[0]
    sp = g.aim_rcs(ctx, Xp, th, ph)[0]
    out["rcs_seconds"] = time.perf_counter() - t0
    mie = [g.mie_sigma_thth(radius, th, ph), g.mie_sigma_thth(radius, th, ph - np.pi / 2)][:npair]
    em = [float(g.err_thth(sm[b], mie[b], w)) for b in range(npair)]
    ep = [float(g.err_thth(sp[b], mie[b], w)) for b in range(npair)]
    out["rcs_directions"] = int(len(th))
    out["err_thth_vs_mie"] = {"mixed": em, "plain": ep, "pols": ["x", "y"][:npair]}
    out["err_thth_mixed_vs_plain"] = [float(g.err_thth(sm[b], sp[b], w)) for b in range(npair)]
    out["equal_accuracy"] = bool(all(a <= b + 1e-3 for a, b in zip(em, ep)))
    g.aim_destroy(ctx)
    del V, Xm, Xp
    torch.cuda.empty_cache()
    return out


def serve_summary(requests=24, slots=4):
    """The small serving stream (plates 1-4 lambda EFIE, spheres 0.5-1 lambda CFIE,
    1-16 RHS): capacity closed-loop, then Poisson arrivals (seed 1) at 0.7 x capacity."""
    from paper_1010_1456_gb300 import serve

    plates, spheres = SERVE_SIZES["small"]
    cap_reqs = serve.make_stream(requests, rate=1.0, seed=2, plate_sides=plates, sphere_radii=spheres,
                                 max_rhs=16, sphere_cfie_alpha=0.6)
    cap_srv = serve.Server(slots=slots)
    res, span = cap_srv.run(cap_reqs, realtime=False)
    cap_srv.close()
    cap = serve.summarize(res, span)
    rate = 0.7 * cap["solves_per_s"]
    reqs = serve.make_stream(requests, rate=rate, seed=1, plate_sides=plates, sphere_radii=spheres, max_rhs=16,
                             sphere_cfie_alpha=0.6)
    srv = serve.Server(slots=slots)
    res, span = srv.run(reqs, realtime=True)
    srv.close()
    summ = serve.summarize(res, span)
    return {"stream": f"plates {plates} lambda (EFIE), spheres {spheres} lambda (CFIE alpha 0.6), 1..16 RHS, "
                      f"{requests} requests, Poisson seed 1 at 0.7 x capacity, {slots} slots",
            "solves_per_s": summ["solves_per_s"], "p50_s": summ["p50_s"], "p99_s": summ["p99_s"],
            "capacity_solves_per_s": cap["solves_per_s"], "failed": summ["failed"],
            "max_rel_res": summ["max_rel_res"], "peak_concurrent": srv.peak_busy,
            "contexts_built": summ["setups"], "mean_requests_per_solve": summ["mean_batch"],
            "batching": "resident contexts per scatterer; queued same-scatterer requests merged into one solve"}


# a catalogue of small scatterers for the multi-instance serving measurement
PACK_CATALOGUE = ((0.8, 0.9, 1.0, 1.1, 1.2), (0.4, 0.45, 0.5, 0.55, 0.6))


def pack_serve_summary(requests=96, slots=2, pack=8):
    """Many small scatterers: a catalogue of five plates (0.8-1.2 lambda, EFIE)
    and five spheres (0.4-0.6 lambda, CFIE alpha 0.6), 1..4 RHS per request,
    contexts resident (built by a warm-up stream), served without and with
    multi-instance packs: closed-loop capacity (seed 2), then Poisson arrivals
    (seed 1) at 0.7 x the capacity without packs, the same stream for both."""
    from paper_1010_1456_gb300 import serve

    plates, spheres = PACK_CATALOGUE

    def stream(seed, rate):
        return serve.make_stream(requests, rate=rate, seed=seed, plate_sides=plates, sphere_radii=spheres, max_rhs=4,
                                 sphere_cfie_alpha=0.6)

    servers, cap = {}, {}
    for name, p in (("without_packs", 1), ("with_packs", pack)):
        srv = serve.Server(slots=slots, pack=p)
        srv.run(stream(5, 1.0), realtime=False)  # builds the resident contexts
        srv.packs = []
        res, span = srv.run(stream(2, 1.0), realtime=False)
        cap[name] = (serve.summarize(res, span), list(srv.packs))
        servers[name] = srv
    rate = 0.7 * cap["without_packs"][0]["solves_per_s"]
    out = {"stream": f"plates {plates} lambda (EFIE), spheres {spheres} lambda (CFIE alpha 0.6), 1..4 RHS, "
                     f"{requests} requests, contexts resident; Poisson seed 1 at {rate:.1f}/s (0.7 x capacity "
                     f"without packs), {slots} slots, packs of up to {pack} scatterers"}
    for name, srv in servers.items():
        srv.packs = []
        res, span = srv.run(stream(1, rate), realtime=True)
        summ = serve.summarize(res, span)
        c, cpacks = cap[name]
        out[name] = {"capacity_solves_per_s": c["solves_per_s"],
                     "capacity_scatterers_per_packed_solve": float(np.mean(cpacks)) if cpacks else None,
                     "solves_per_s": summ["solves_per_s"], "p50_s": summ["p50_s"], "p99_s": summ["p99_s"],
                     "failed": summ["failed"], "max_rel_res": summ["max_rel_res"],
                     "mean_requests_per_solve": summ["mean_batch"],
                     "scatterers_per_packed_solve": float(np.mean(srv.packs)) if srv.packs else None}
        srv.close()
    return out


# ---------------------------------------------------------------- serving
SERVE_SIZES = {
    # the stream of the serving configuration: plate sides / sphere radii in wavelengths
    "paper": ((2, 4, 8, 16, 32), (1, 2, 4, 8)),
    "small": ((1, 2, 4), (0.5, 1)),
}


def run_serve(args):
    """Continuous-batching stream: capacity (closed loop), then Poisson arrivals at 0.7 x capacity."""
    import torch

    from paper_1010_1456_gb300 import serve

    torch.cuda.set_device(0)
    plates, spheres = SERVE_SIZES[args.serve_sizes]
    cap_reqs = serve.make_stream(args.requests, rate=1.0, seed=2, plate_sides=plates, sphere_radii=spheres,
                                 max_rhs=args.serve_max_rhs, sphere_cfie_alpha=args.serve_cfie)
    srv = serve.Server(slots=args.slots, cache=bool(args.serve_cache))
    res, span = srv.run(cap_reqs, realtime=False)
    srv.close()
    cap = serve.summarize(res, span)
    rate = 0.7 * cap["solves_per_s"]
    reqs = serve.make_stream(args.requests, rate=rate, seed=1, plate_sides=plates, sphere_radii=spheres,
                             max_rhs=args.serve_max_rhs, sphere_cfie_alpha=args.serve_cfie)
    srv = serve.Server(slots=args.slots, cache=bool(args.serve_cache))
    t0 = time.perf_counter()
    with ClockSampler(0) as clk:
        res, span = srv.run(reqs, realtime=True)
    wall = time.perf_counter() - t0
    srv.close()
    summ = serve.summarize(res, span)
    line = {
        "metric": "served solves/s (p50/p99 latency), complex64 AIM with FP64 refinement, tol 1e-6",
        "value": summ["solves_per_s"],
        "unit": "solves/s",
        "n_gpus": 1,
        "higher_is_better": True,
        "data": "synthetic",
        "config": {"workload": f"serving stream ({args.serve_sizes} sizes): plates {plates} lambda (EFIE), spheres "
                               f"{spheres} lambda ({'CFIE alpha %g' % args.serve_cfie if args.serve_cfie < 1 else 'EFIE'}), "
                               f"1..{args.serve_max_rhs} RHS, Poisson seed 1 at 0.7 x capacity",
                   "requests": args.requests, "slots": args.slots},
        "p50_s": summ["p50_s"],
        "p99_s": summ["p99_s"],
        "rhs_per_s": summ["rhs_per_s"],
        "capacity_solves_per_s": cap["solves_per_s"],
        "arrival_rate_per_s": rate,
        "failed": summ["failed"],
        "max_rel_res": summ["max_rel_res"],
        "peak_concurrent": srv.peak_busy,
        "contexts_built": summ["setups"],
        "mean_requests_per_solve": summ["mean_batch"],
        "resident_contexts": bool(args.serve_cache),
        "wall_s": wall,
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- complexity sweep
SWEEP = {"plate": (1, 2, 4, 8, 16, 32, 64), "sphere": (1, 2, 4, 8, 16)}


def run_sweep(args):
    """Matvec time against N over the plates 1-64 lambda and spheres 1-16 lambda
    (the shape of the paper's complexity figure, Section 3, on one GPU): one
    right-hand side, complex64 and FP64-accurate products, FFT kernels
    autotuned, L2 flushed between products."""
    import torch

    import paper_1010_1456_gb300 as g

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    rows = []
    from aim_inputs import random_complex

    kinds = [(k, sz) for k in ("plate", "sphere") for sz in SWEEP[k] if not args.sweep_max or sz <= args.sweep_max]
    for kind, size in kinds:
        verts, tris = mesh_for(kind, size)
        t0 = time.perf_counter()
        ctx = g.aim_setup(verts, tris, K0, H, M=2, near_radius=3 * H, max_rhs=1, stream=stream.cuda_stream)
        setup_s = time.perf_counter() - t0
        n, L, nnz = g.aim_grid_info(ctx)
        row = {"kind": kind, "size_lambda": size, "N": ctx.N, "grid": n, "padded": L, "nnz_near": nnz,
               "setup_s": round(setup_s, 3)}
        xh = random_complex((1, ctx.N), 7)
        for name, P, dt in (("c64", g.AIM_C64, torch.complex64), ("fp64_accurate", g.AIM_C128, torch.complex128)):
            x = torch.from_numpy(xh).to(dev, dt)
            y = torch.empty_like(x)
            g.aim_autotune(ctx, P, nrhs=1, reps=2)
            for _ in range(3):
                g.aim_matvec(ctx, x, y, precision=P)
            torch.cuda.synchronize()
            reps = 20
            tot = 0.0
            for _ in range(reps):
                flush.zero_()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                g.aim_matvec(ctx, x, y, precision=P)
                b.record(stream)
                torch.cuda.synchronize()
                tot += a.elapsed_time(b)
            row[name + "_ms"] = round(tot / reps, 4)
        rows.append(row)
        ctx.close()
        del ctx
        torch.cuda.empty_cache()
    line = {"metric": "AIM matvec time vs N (complexity sweep)", "unit": "ms", "n_gpus": 1, "data": "synthetic",
            "config": {"workload": "PEC plates 1-64 lambda (mesh lambda/9) and icospheres 1-16 lambda, h = lambda/10, "
                                   "M = 2, near radius 3h, one RHS", "l2": "flushed between products"},
            "rows": rows}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- reference arm
def run_reference(args, rank, world):
    """The oracle on this host's cores for the same workload: every step is one
    bounded piece (a quarter of one right-hand side's product, OracleSample)."""
    if rank != 0:
        return 0
    from aim_inputs import random_complex

    kind, size, nrhs, prec = WORKLOADS[args.workload]
    verts, tris = mesh_for(kind, size)
    o = OracleSample(verts, tris)
    x = random_complex((1, o.N), 1)
    for _ in range(args.warmup):
        o.piece(x)
    for _ in range(args.steps):
        o.piece(x)
    base = o.result(warm=args.warmup)
    line = {
        "impl": "reference",
        "metric": METRIC,
        "value": base["value"],
        "unit": "matvec/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": float(np.mean(o.t[args.warmup:]) * 1e3),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": args.workload, "nrhs": nrhs,
                   "step": "a quarter of one right-hand side's product (one grid component) on the host"},
        "cpu_baseline": base,
        "e2e": {"value": base["value"], "unit": "matvec/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- our arm
FFT_KERNEL_NAMES = {1: "stockham", 2: "fourstep", 3: "fourstep_small", 4: "fourstep_warp", 5: "fourstep_wide"}


def fft_kernel_names(g, chosen, L):
    """Pass -> kernel name; a planar grid (L_z = 1) runs no z passes."""
    return {p_: ("none (planar grid)" if L[2] == 1 and p_ in ("fft_z_fwd", "fft_z_inv") else FFT_KERNEL_NAMES[k])
            for p_, k in zip(g.FFT_PASSES, chosen)}


def cufft_comparison(torch, dev, stream, L, nrhs, wide, kernels, flush, reps=5, max_gb=8.0):
    """Timed comparison only: the same convolution on the full zero-padded grids
    through cuFFT (torch.fft: forward 3-D FFT, product with a spectrum, inverse),
    against the five pruned passes of this library."""
    G = 4 * nrhs
    dt = torch.complex128 if wide else torch.complex64
    esize = 16 if wide else 8
    gb = G * int(np.prod(L)) * esize / 1e9
    ours = sum(kernels[k]["avg_ms"] for k in ("fft_z_fwd", "fft_y_fwd", "fft_x_conv", "fft_y_inv", "fft_z_inv")
               if k in kernels)
    if gb > max_gb:
        return {"skipped": f"padded batch of {gb:.1f} GB (> {max_gb} GB)", "ours_fft_ms": ours}
    Lx, Ly, Lz = L
    a = torch.randn(G, Lz, Ly, Lx, dtype=dt, device=dev)
    spec = torch.randn(Lz, Ly, Lx, dtype=dt, device=dev)
    for _ in range(3):
        torch.fft.ifftn(torch.fft.fftn(a, dim=(1, 2, 3)) * spec, dim=(1, 2, 3))
    torch.cuda.synchronize()
    tot = 0.0
    for _ in range(reps):
        flush.zero_()
        b, e_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        b.record(stream)
        torch.fft.ifftn(torch.fft.fftn(a, dim=(1, 2, 3)) * spec, dim=(1, 2, 3))
        e_.record(stream)
        torch.cuda.synchronize()
        tot += b.elapsed_time(e_)
    del a, spec
    torch.cuda.empty_cache()
    return {"what": "cuFFT (torch.fft) forward + spectral product + inverse on the unpruned padded grids",
            "cufft_ms": tot / reps, "ours_fft_ms": ours, "speedup_ours": (tot / reps) / ours if ours else None}


def time_products(g, torch, ctx, x, y, P, steps, stream, flush):
    """Mean ms of `steps` products (CUDA events on the context stream, L2 flushed between them)."""
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for i in range(steps):
        flush.zero_()
        evs[i][0].record(stream)
        g.aim_matvec(ctx, x, y, precision=P)
        evs[i][1].record(stream)
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in evs) / steps


def plain_single_rhs_products(g, torch, verts, tris, xh, stream, flush, autotune, steps=10):
    """The plain single-RHS FP64 path: FP64-accurate (float-float) and native
    FP64 products of one vector on a one-RHS context."""
    dev = flush.device
    ctx1 = g.aim_setup(verts, tris, K0, H, M=2, near_radius=3 * H, max_rhs=1, precision=g.AIM_C128,
                       stream=stream.cuda_stream)
    x1 = torch.from_numpy(xh[:1].astype(np.complex128)).to(dev)
    y1 = torch.empty_like(x1)
    out = {}
    for name, VP, what in (("fp64_accurate", g.AIM_C128, "float-float arithmetic end to end (FP64-accurate)"),
                           ("native_fp64", g.AIM_C128_F64, "native FP64 arithmetic end to end")):
        if autotune:
            g.aim_autotune(ctx1, VP, nrhs=1, reps=2)
        for _ in range(3):
            g.aim_matvec(ctx1, x1, y1, precision=VP)
        torch.cuda.synchronize()
        ms = time_products(g, torch, ctx1, x1, y1, VP, steps if VP == g.AIM_C128 else max(3, steps // 3), stream,
                           flush)
        out[name] = {"what": what, "matvec_per_s": 1e3 / ms, "ms_per_product": ms}
    ctx1.close()
    del x1, y1
    torch.cuda.empty_cache()
    return out


def run_ours(args, rank, world, local_rank):
    import torch

    import paper_1010_1456_gb300 as g
    from aim_inputs import random_complex

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    kind, size, nrhs, prec = WORKLOADS[args.workload]
    verts, tris = mesh_for(kind, size)
    P = PRECISION[prec]
    wide = prec != "c64"
    e = 16 if wide else 8
    stream = torch.cuda.current_stream(dev)
    t0 = time.perf_counter()
    ctx = g.aim_setup(verts, tris, K0, H, M=2, near_radius=3 * H, max_rhs=nrhs, precision=P,
                      stream=stream.cuda_stream)
    setup_s = time.perf_counter() - t0
    n, L, nnz = g.aim_grid_info(ctx)
    N = ctx.N

    xh = random_complex((nrhs, N), 1000 + rank).astype(np.complex128 if wide else np.complex64)
    x = torch.from_numpy(xh).to(dev)
    y = torch.empty_like(x)
    tune = None
    if args.autotune:
        t0 = time.perf_counter()
        chosen, tune_ms = g.aim_autotune(ctx, P, nrhs=nrhs, reps=3)
        tune = {"seconds": round(time.perf_counter() - t0, 2),
                "kernels": fft_kernel_names(g, chosen, L),
                "pass_ms": {p_: {FFT_KERNEL_NAMES[k]: round(float(tune_ms[i, k]), 4) for k in FFT_KERNEL_NAMES
                                 if tune_ms[i, k] > 0} for i, p_ in enumerate(g.FFT_PASSES)}}
    else:
        chosen = g.aim_fft_config(ctx, P)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    for _ in range(args.warmup):
        g.aim_matvec(ctx, x, y, precision=P)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    g.aim_profile(ctx, 2)
    g.aim_profile(ctx, 1)
    l0 = g.aim_launch_count(ctx)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local_rank) as clk:
        for i in range(args.steps):
            flush.zero_()  # L2 flush between timed products, outside the events
            ev[i][0].record(stream)
            g.aim_matvec(ctx, x, y, precision=P)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
    launches = g.aim_launch_count(ctx) - l0
    g.aim_profile(ctx, 0)
    prof = g.aim_profile_read(ctx)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms, value = aggregate(sum(step_ms), args.steps, nrhs, world, dev)

    # end to end through the host-buffer entry point (copies inside the timed region)
    e2e_steps = max(3, min(args.steps, 10))
    xp = torch.from_numpy(xh).pin_memory()  # pinned host buffers: the copies run at full link speed
    yp = torch.empty_like(xp).pin_memory()
    g.aim_matvec_host(ctx, xp, precision=P, out=yp)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        g.aim_matvec_host(ctx, xp, precision=P, out=yp)
    e2e_s = time.perf_counter() - t0
    e2e = {"value": world * e2e_steps * nrhs / e2e_s, "unit": "matvec/s", "host_buffers": "pinned",
           "h2d_bytes_per_step": int(xh.nbytes), "d2h_bytes_per_step": int(xh.nbytes), "steps": e2e_steps}
    del xp, yp

    # roofline of the dominant kernel: the method's algorithmic bytes per launch (pass model)
    pptr = g.aim_export(ctx, g.AIM_EXPORT_PROJ_PTR)
    nent = int(pptr[-1])
    cnt = np.diff(pptr)
    touched = int(np.count_nonzero(cnt))
    # a grid with z passes is projected over its 8-node groups with entries
    # (fewer than 16 RHS; the many-RHS projection writes every node)
    groups = int(np.count_nonzero(np.add.reduceat(cnt, np.arange(0, len(cnt), 8))))
    projected = 8 * groups if (L[2] > 1 and nrhs < 16) else None
    S = 9 if L[2] == 1 else 27  # stencil nodes (M = 2; a planar grid keeps one plane)
    models = kernel_models(N, n, L, nnz, nent, S, nrhs, e, touched, projected)
    tot_ms = max(sum(v[1] for v in prof.values()), 1e-30)
    kernels = {k: {"launches": c, "avg_ms": ms / max(c, 1), "share": ms / tot_ms} for k, (c, ms) in prof.items()}
    dom = max(kernels, key=lambda k: kernels[k]["share"])
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    hbm = peaks.get("hbm_gbs", 6800.0)
    hbm_src = "MEASURED_PEAKS.json hbm_gbs (measured)" if "hbm_gbs" in peaks else "fallback 6.8 TB/s"
    alu64 = g.aim_probe_fma_peak(64)
    alu32 = g.aim_probe_fma_peak(32)
    for k, v in kernels.items():
        if k in models:
            b, f = models[k]
            s_ = v["avg_ms"] * 1e-3
            v["GB/s"] = b / s_ / 1e9
            v["hbm_frac"] = b / s_ / 1e9 / hbm
            v["TFLOP/s"] = f / s_ / 1e12
    roof = None
    if dom in models:
        bytes_, flops = models[dom]
        avg_s = kernels[dom]["avg_ms"] * 1e-3
        roof = {"bound": "hbm", "kernel": dom, "achieved": bytes_ / avg_s / 1e9, "peak": hbm, "unit": "GB/s",
                "frac": bytes_ / avg_s / 1e9 / hbm, "peak_source": hbm_src, "traffic": ncu_traffic(args.workload, dom),
                "algorithmic_bytes": bytes_, "avg_launch_ms": kernels[dom]["avg_ms"],
                "bytes_model": "pass model: G = 4 x nrhs grids; x pass reads and writes G Lz Ly nx complex values "
                               "plus the Ghat octant; strided passes read n_in and write n_out samples per pencil"}
        if prec == "c128":
            ff32 = ff_fft_flops(dom, n, L, nrhs)
            if ff32 is not None:
                roof["fp32_issue"] = {"achieved_tflops": ff32 / avg_s / 1e12, "peak_tflops": alu32,
                                      "frac": ff32 / avg_s / 1e12 / alu32,
                                      "counts": "FP32 flops of the float-float butterflies (ff_fft_flops)"}
        else:
            roof["fp32_issue"] = {"achieved_tflops": flops / avg_s / 1e12, "peak_tflops": alu32 if prec == "c64"
                                  else alu64, "frac": flops / avg_s / 1e12 / (alu32 if prec == "c64" else alu64),
                                  "counts": "5 L log2 L flops per length-L transform (+ the spectral product)"}
        roof["all_kernels_hbm_frac"] = sum(models[k][0] for k in kernels if k in models) / (
            sum(kernels[k]["avg_ms"] for k in kernels if k in models) * 1e-3) / 1e9 / hbm

    variants = None
    if args.variants:
        if nrhs > 1:
            variants = plain_single_rhs_products(g, torch, verts, tris, xh, stream, flush, args.autotune)
        else:
            variants = {}
            for vname, VP in (("native_fp64", g.AIM_C128_F64), ("fp64_accurate", g.AIM_C128), ("c64", g.AIM_C64)):
                if VP == P:
                    continue
                xv = torch.from_numpy(xh.astype(np.complex64 if VP == g.AIM_C64 else np.complex128)).to(dev)
                yv = torch.empty_like(xv)
                if args.autotune:
                    g.aim_autotune(ctx, VP, nrhs=nrhs, reps=3)
                for _ in range(3):
                    g.aim_matvec(ctx, xv, yv, precision=VP)
                torch.cuda.synchronize()
                ms = time_products(g, torch, ctx, xv, yv, VP, max(10, args.steps // 4), stream, flush)
                variants[vname] = {"matvec_per_s": nrhs * 1e3 / ms, "ms_per_product": ms}
                del xv, yv
    cufft = cufft_comparison(torch, dev, stream, L, nrhs, wide, kernels, flush) if args.cufft else None
    ctx.close()
    del ctx, x, y
    torch.cuda.empty_cache()

    solve = None
    if args.solve:
        if kind == "sphere":
            solve = solve_section_sphere(g, verts, tris, size, nrhs, stream)
        else:
            c2 = g.aim_setup(verts, tris, K0, H, M=2, near_radius=3 * H, max_rhs=nrhs, precision=P,
                             stream=stream.cuda_stream)
            solve = solve_section(g, c2, kind, size, nrhs, P)
            c2.close()
            torch.cuda.empty_cache()
    serving = serve_summary() if args.serve_extra else None
    serving_packs = pack_serve_summary() if args.serve_extra else None

    line = {
        "metric": METRIC,
        "value": value,
        "unit": "matvec/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": {"f64": "f64", "c128": "f64 in and out, float-float (f32 pairs) throughout", "c64": "c64 (f32)"}[prec],
        "data": "synthetic",
        "config": {"workload": args.workload, "N": N, "grid": n, "padded": L, "nnz_near": nnz, "nrhs": nrhs,
                   "formulation": "EFIE", "M": 2, "h_lambda": H, "near_radius_h": 3,
                   "l2": "inputs (60 GB of grids at the 16 lambda sphere) exceed L2; also flushed between steps "
                         "(256 MB write)",
                   "parallelism": f"replicas x{world}", "setup_s": round(setup_s, 2),
                   "fft_kernels": fft_kernel_names(g, chosen, L)},
        "roofline": roof,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clk.summary(),
        "plain_fp64_single_rhs": variants if nrhs > 1 else None,
        "variants": variants if nrhs == 1 else None,
        "solve": solve,
        "serving": serving,
        "serving_many_small_scatterers": serving_packs,
        "autotune": tune,
        "cufft_comparison": cufft,
        "kernels": kernels,
        "fp64_fma_tflops": alu64,
        "fp32_fma_tflops": alu32,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = oracle_matvec_rate(verts, tris, budget_s=args.cpu_budget)
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default=DEFAULT)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--solve", type=int, default=1, help="1: also time plain and mixed solves")
    ap.add_argument("--variants", type=int, default=1, help="1: also time the other product precisions")
    ap.add_argument("--autotune", type=int, default=1, help="1: autotune the FFT kernels before timing")
    ap.add_argument("--cufft", type=int, default=1, help="1: also time the unpruned cuFFT convolution (grids <= 8 GB)")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--serve-extra", type=int, default=1, help="1: add the small serving stream's p50/p99")
    ap.add_argument("--serve", action="store_true", help="run the serving stream instead of the product benchmark")
    ap.add_argument("--sweep", action="store_true", help="matvec time against N over plates and spheres")
    ap.add_argument("--sweep-max", type=float, default=0.0, help="largest size (lambda) in the sweep; 0: all")
    ap.add_argument("--serve-sizes", choices=sorted(SERVE_SIZES), default="small")
    ap.add_argument("--requests", type=int, default=40)
    ap.add_argument("--slots", type=int, default=4)
    ap.add_argument("--serve-max-rhs", type=int, default=16)
    ap.add_argument("--serve-cache", type=int, default=1,
                    help="1: resident contexts and merged same-scatterer solves; 0: one context per request")
    ap.add_argument("--serve-cfie", type=float, default=0.6,
                    help="alpha of the CFIE the spheres of the serving stream are solved with (1: EFIE)")
    args = ap.parse_args()
    if args.sweep:
        return run_sweep(args)
    if args.serve:
        return run_serve(args)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if world > 1:
        import torch

        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    try:
        return run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch

            torch.distributed.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
