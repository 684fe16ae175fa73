"""Continuous-batching request loop for AIM scattering solves.

Each request is one scatterer (mesh, wavenumber, excitation set) to be solved
with FP64-refined complex64 AIM (``aim_solve`` with AIM_C64).  The server
keeps ``slots`` worker threads, each with its own CUDA stream.  A request is
admitted as soon as a slot is free and its estimated device footprint
(``aim_footprint``) fits in the memory budget that the running requests have
not claimed; admission is in arrival order, but a request that does not fit
does not block later requests that do (up to ``max_skip`` passes).  Admitted
requests run concurrently: their setup (host), spectra, products and Krylov
steps interleave on the device.  The library calls release the GIL, so the
threads overlap.

The request/response path is the library's C ABI only; no step of a solve
runs in Python.
"""

import dataclasses
import queue
import threading
import time

import numpy as np

from . import (
    AIM_C64,
    aim_footprint,
    aim_rcs,
    aim_rhs_planewave,
    aim_setup,
    aim_solve,
)


@dataclasses.dataclass
class Request:
    rid: int
    verts: np.ndarray
    tris: np.ndarray
    khat: np.ndarray  # [nrhs, 3]
    pol: np.ndarray  # [nrhs, 3]
    k: float = 2 * np.pi
    h: float = 0.1
    M: int = 2
    near_radius: float = 0.3
    tol: float = 1e-6
    arrival: float = 0.0  # seconds after the stream start
    rcs_dirs: tuple = None  # optional (theta, phi) arrays
    label: str = ""
    cfie_alpha: float = 1.0  # < 1: CFIE (closed bodies only)


@dataclasses.dataclass
class Result:
    rid: int
    X: np.ndarray
    rel_res: np.ndarray
    iterations: int
    arrival: float
    admitted: float
    finished: float
    footprint: int
    sigma: np.ndarray = None
    error: str = None

    @property
    def latency(self):
        return self.finished - self.arrival


class Server:
    def __init__(self, slots=4, mem_budget=None, device=0, precision=AIM_C64, max_skip=8):
        import torch

        self.torch = torch
        self.device = device
        if mem_budget is None:
            torch.cuda.set_device(device)
            free, _total = torch.cuda.mem_get_info(device)
            mem_budget = int(0.8 * free)
        self.budget = int(mem_budget)
        self.peak_claimed = 0
        self.peak_busy = 0
        self.slots = slots
        self.precision = precision
        self.max_skip = max_skip
        self.claimed = 0
        self.lock = threading.Condition()
        self.pending = []  # admitted-not-yet requests, arrival order
        self.results = {}
        self.busy = 0
        self.stop = False
        self.t0 = None

    # -------------------------------------------------------------- admission
    def _admissible(self):
        """Pop the first pending request that fits (under the lock)."""
        for i, (req, fp) in enumerate(self.pending[: self.max_skip]):
            if self.claimed + fp <= self.budget or (self.busy == 0 and self.claimed == 0):
                self.pending.pop(i)
                return req, fp
        return None

    def _make_stream(self):
        torch = self.torch
        torch.cuda.set_device(self.device)
        return torch.cuda.Stream(self.device)

    def _worker(self, wid):
        stream = self._make_stream()
        while True:
            with self.lock:
                while True:
                    if self.stop and not self.pending:
                        return
                    got = self._admissible() if self.pending else None
                    if got is not None:
                        req, fp = got
                        self.claimed += fp
                        self.busy += 1
                        self.peak_claimed = max(self.peak_claimed, self.claimed)
                        self.peak_busy = max(self.peak_busy, self.busy)
                        break
                    self.lock.wait(0.05)
            admitted = time.perf_counter() - self.t0
            res = self._run(req, fp, stream, admitted)
            with self.lock:
                self.claimed -= fp
                self.busy -= 1
                self.results[req.rid] = res
                self.lock.notify_all()

    def _run(self, req, fp, stream, admitted):
        torch = self.torch
        try:
            with torch.cuda.stream(stream):
                nrhs = len(req.khat)
                ctx = aim_setup(req.verts, req.tris, req.k, req.h, M=req.M, near_radius=req.near_radius,
                                precision=self.precision, max_rhs=nrhs, stream=stream.cuda_stream,
                                cfie_alpha=req.cfie_alpha)
                try:
                    V = aim_rhs_planewave(ctx, req.khat, req.pol)
                    X, info = aim_solve(ctx, V, req.tol, raise_on_noconv=False)
                    sigma = None
                    if req.rcs_dirs is not None:
                        sigma = aim_rcs(ctx, X, *req.rcs_dirs)[0]
                    Xh = X.cpu().numpy()
                finally:
                    ctx.close()
            return Result(req.rid, Xh, info["rel_res"], info["iterations"], req.arrival, admitted,
                          time.perf_counter() - self.t0, fp, sigma)
        except Exception as e:  # reported per request; the server keeps running
            return Result(req.rid, None, None, 0, req.arrival, admitted, time.perf_counter() - self.t0, fp,
                          error=repr(e))

    def _footprint(self, req):
        return aim_footprint(req.verts, req.tris, req.h, req.M, req.near_radius, len(req.khat), req.cfie_alpha,
                             self.precision)

    # -------------------------------------------------------------- driver
    def run(self, requests, realtime=True):
        """Feed requests at their arrival times (or all at once) and wait for all results."""
        self.t0 = time.perf_counter()
        threads = [threading.Thread(target=self._worker, args=(i,), daemon=True) for i in range(self.slots)]
        for t in threads:
            t.start()
        for req in sorted(requests, key=lambda r: r.arrival):
            if realtime:
                dt = req.arrival - (time.perf_counter() - self.t0)
                if dt > 0:
                    time.sleep(dt)
            fp = self._footprint(req)
            with self.lock:
                self.pending.append((req, fp))
                self.lock.notify_all()
        with self.lock:
            self.stop = True
            self.lock.notify_all()
        for t in threads:
            t.join()
        makespan = time.perf_counter() - self.t0
        return [self.results[r.rid] for r in requests], makespan


def summarize(results, makespan):
    lat = np.array([r.latency for r in results if r.error is None])
    ok = [r for r in results if r.error is None]
    return {
        "solves": len(ok),
        "failed": len(results) - len(ok),
        "solves_per_s": len(ok) / makespan if makespan > 0 else 0.0,
        "p50_s": float(np.percentile(lat, 50)) if len(lat) else None,
        "p99_s": float(np.percentile(lat, 99)) if len(lat) else None,
        "rhs_per_s": sum(len(r.X) for r in ok) / makespan if makespan > 0 else 0.0,
        "makespan_s": makespan,
        "max_rel_res": float(max(r.rel_res.max() for r in ok)) if ok else None,
    }


def make_stream(n_requests, rate, seed=1, plate_sides=(2, 4, 8, 16, 32), sphere_radii=(1, 2, 4, 8), max_rhs=16,
                theta_max_deg=80.0, sphere_cfie_alpha=1.0):
    """Synthetic request stream: Poisson arrivals at ``rate`` per second.

    Draw order per request: inter-arrival time, kind (plate or sphere, 50/50),
    size, number of right-hand sides (uniform 1..max_rhs), then the incidence
    angles and polarisations (``aim_inputs.random_incidence``).  Spheres are
    solved with CFIE when ``sphere_cfie_alpha`` < 1 (Section 2.2 uses 0.6 for
    closed bodies); plates are open and always take the EFIE.
    """
    from aim_inputs import icosphere_frequency, icosphere_mesh, plate_mesh, random_incidence

    rng = np.random.default_rng(seed)
    t = 0.0
    reqs = []
    cache = {}
    for i in range(n_requests):
        t += rng.exponential(1.0 / rate)
        plate = rng.uniform() < 0.5
        size = float(rng.choice(plate_sides if plate else sphere_radii))
        nrhs = int(rng.integers(1, max_rhs + 1))
        ndir = (nrhs + 1) // 2
        kh, po = random_incidence(ndir, theta_max_deg=theta_max_deg, rng=rng)
        kh, po = kh[:nrhs], po[:nrhs]
        key = (plate, size)
        if key not in cache:
            cache[key] = plate_mesh(size, int(round(9 * size))) if plate else icosphere_mesh(size, icosphere_frequency(size))
        v, tr = cache[key]
        reqs.append(Request(i, v, tr, kh, po, arrival=t, label=f"{'plate' if plate else 'sphere'}{size:g}x{nrhs}",
                            cfie_alpha=1.0 if plate else float(sphere_cfie_alpha)))
    return reqs
