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

Two batching levels sit on top (``cache=True``, the default):

* resident contexts: a context built for a scatterer (mesh, k, h, M, near
  radius, CFIE alpha, tolerance) stays on the device after its solve, so a
  later request for the same scatterer skips the setup; idle contexts are
  evicted least recently used when the memory budget needs room;
* merged solves: when a slot takes a request, every pending request for the
  same scatterer joins it (up to ``merge_rhs`` right-hand sides in total) and
  the group is solved as one multi-RHS solve, so each product, FFT pass and
  Krylov step is one launch for all of them.  Each right-hand side keeps its
  own Arnoldi process in the batched GMRES, so a request's result is the one
  it would get alone.

A third level packs different scatterers (``pack`` > 1): a slot that takes a
request also takes pending requests for other scatterers of the same pack
class (k, h, M, tolerance, flat or not; see ``pack_class``) whose grid boxes
are within ``pack_ratio`` of the first one's volume, up to ``pack`` scatterers
and ``pack_rhs`` right-hand sides, and solves them as one multi-instance pack
(``aim_pack_create`` / ``aim_pack_solve``): every product stage is one launch
for all of them, and each right-hand side keeps its own Arnoldi process.

The request/response path is the library's C ABI only; no step of a solve
runs in Python.
"""

import dataclasses
import hashlib
import threading
import time

import numpy as np

from . import (
    AIM_C64,
    AIMError,
    aim_footprint,
    aim_pack_create,
    aim_pack_solve,
    aim_rcs,
    aim_rhs_planewave,
    aim_set_stream,
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
    batch: int = 1  # requests solved together in this request's solve
    setup: bool = True  # a context was built for this result (the first request of a batch that found none)

    @property
    def latency(self):
        return self.finished - self.arrival


def scatterer_key(req):
    """Requests with equal keys share one operator: same mesh, wavenumber, grid
    step, stencil order, near radius, CFIE weight and tolerance."""
    h = hashlib.sha1()
    h.update(np.ascontiguousarray(req.verts, dtype=np.float64).tobytes())
    h.update(np.ascontiguousarray(req.tris, dtype=np.int32).tobytes())
    return (h.hexdigest(), float(req.k), float(req.h), int(req.M), float(req.near_radius), float(req.cfie_alpha),
            float(req.tol))


def pack_class(req):
    """Requests whose contexts can share a pack: equal k, h, M and tolerance, and
    the same grid layout (a mesh flat in z gets the planar grid)."""
    flat = bool(np.ptp(np.asarray(req.verts)[:, 2]) == 0.0)
    return (float(req.k), float(req.h), int(req.M), float(req.tol), flat)


def box_volume(req):
    """Nodes of the request's grid box, estimated from the mesh's bounding box."""
    v = np.asarray(req.verts)
    n = np.floor(np.ptp(v, axis=0) / req.h) + req.M + 2
    if np.ptp(v[:, 2]) == 0.0:
        n[2] = 1
    return float(np.prod(n))


class Server:
    def __init__(self, slots=4, mem_budget=None, device=0, precision=AIM_C64, max_skip=8, cache=True,
                 merge_rhs=16, pack=1, pack_rhs=64, pack_ratio=4.0):
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
        self.cache = cache
        self.merge_rhs = int(merge_rhs)
        self.pack = int(pack) if cache else 1  # packs are built from resident contexts
        self.pack_rhs = int(pack_rhs)
        self.pack_ratio = float(pack_ratio)
        self.packs = []  # scatterers per packed solve
        self.claimed = 0  # footprints of running uncached requests and of every resident context
        self.lock = threading.Condition()
        self.pending = []  # admitted-not-yet requests, arrival order: (req, footprint, key)
        self.results = {}
        self.busy = 0
        self.stop = False
        self.t0 = None
        # resident contexts: key -> {"ctx", "fp", "busy", "used"}
        self.contexts = {}
        self.setups = 0
        self.batches = []  # sizes of the solves run

    # -------------------------------------------------------------- admission
    def _evict_idle(self, need):
        """Free idle resident contexts, least recently used first, until `need` bytes fit (under the lock)."""
        for key, ent in sorted(self.contexts.items(), key=lambda kv: kv[1]["used"]):
            if self.claimed + need <= self.budget:
                break
            if ent["busy"]:
                continue
            ent["ctx"].close()
            self.claimed -= ent["fp"]
            del self.contexts[key]

    def _admissible(self):
        """Pop the first pending request that can run now, with the pending requests
        that merge into its solve (under the lock).  Returns (batch, claim) or None;
        claim is the footprint charged for the batch's duration (0 when it reuses a
        resident context, whose footprint stays claimed while it is resident)."""
        for i, (req, fp, key) in enumerate(self.pending[: self.max_skip]):
            ent = self.contexts.get(key) if self.cache else None
            if ent is not None and ent["busy"]:
                continue  # its context is solving: this request waits for it (or merges into the next solve)
            need = 0 if ent is not None else fp
            if self.cache and need and self.claimed + need > self.budget:
                self._evict_idle(need)
            if need == 0 or self.claimed + need <= self.budget or (self.busy == 0 and self.claimed == 0):
                self.pending.pop(i)
                batch = [req]
                if self.cache:
                    tot = len(req.khat)
                    j = 0
                    while j < len(self.pending):
                        r2, _fp2, k2 = self.pending[j]
                        if k2 == key and tot + len(r2.khat) <= self.merge_rhs:
                            batch.append(r2)
                            tot += len(r2.khat)
                            self.pending.pop(j)
                        else:
                            j += 1
                    if ent is None:  # the context this solve builds stays resident
                        self.contexts[key] = {"ctx": None, "fp": fp, "busy": True, "used": time.perf_counter()}
                    else:
                        ent["busy"] = True
                        ent["used"] = time.perf_counter()
                    if self.pack > 1:
                        need += self._pack_more(req, key, batch, need)
                return batch, need
        return None

    def _pack_more(self, req, key, batch, need):
        """Add to `batch` the pending requests of other scatterers that can share
        its pack (each with its same-scatterer followers); returns the footprint
        their new contexts add to the claim (under the lock)."""
        cls, vol = pack_class(req), box_volume(req)
        keys = {key}
        tot = sum(len(r.khat) for r in batch)
        extra = 0
        j = 0
        while j < len(self.pending) and len(keys) < self.pack:
            r2, fp2, k2 = self.pending[j]
            ent2 = self.contexts.get(k2)
            v2 = box_volume(r2)
            fits = (k2 not in keys and pack_class(r2) == cls and max(v2, vol) <= self.pack_ratio * min(v2, vol)
                    and tot + len(r2.khat) <= self.pack_rhs and not (ent2 is not None and ent2["busy"]))
            need2 = 0 if ent2 is not None else fp2
            if not fits or (need2 and self.claimed + need + extra + need2 > self.budget):
                j += 1
                continue
            self.pending.pop(j)
            group = [r2]
            ntot = len(r2.khat)
            i = j
            while i < len(self.pending):  # its own followers, as for the first scatterer
                r3, _fp3, k3 = self.pending[i]
                if k3 == k2 and ntot + len(r3.khat) <= self.merge_rhs and tot + ntot + len(r3.khat) <= self.pack_rhs:
                    group.append(r3)
                    ntot += len(r3.khat)
                    self.pending.pop(i)
                else:
                    i += 1
            batch.extend(group)
            tot += ntot
            keys.add(k2)
            extra += need2
            if ent2 is None:
                self.contexts[k2] = {"ctx": None, "fp": fp2, "busy": True, "used": time.perf_counter()}
            else:
                ent2["busy"] = True
                ent2["used"] = time.perf_counter()
        return extra

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
                        batch, claim = got
                        self.claimed += claim
                        self.busy += 1
                        self.peak_claimed = max(self.peak_claimed, self.claimed)
                        self.peak_busy = max(self.peak_busy, self.busy)
                        self.batches.append(len(batch))
                        break
                    self.lock.wait(0.05)
            admitted = time.perf_counter() - self.t0
            res = self._solve_batch(batch, claim, stream, admitted)
            with self.lock:
                if not self.cache:
                    self.claimed -= claim
                else:
                    for key in dict.fromkeys(scatterer_key(r) for r in batch):
                        ent = self.contexts.get(key)
                        if ent is not None:
                            ent["busy"] = False
                            ent["used"] = time.perf_counter()
                            if ent["ctx"] is None:  # its setup failed: nothing resident
                                self.claimed -= ent["fp"]
                                del self.contexts[key]
                self.busy -= 1
                for r in res:
                    self.results[r.rid] = r
                self.lock.notify_all()

    def _solve_batch(self, batch, claim, stream, admitted):
        if not self.cache:
            return [self._run(req, self._footprint(req), stream, admitted) for req in batch]
        groups = {}
        for r in batch:
            groups.setdefault(scatterer_key(r), []).append(r)
        if len(groups) > 1:
            return self._run_packed(list(groups.values()), stream, admitted)
        return self._run_merged(batch, stream, admitted)

    def _run(self, req, fp, stream, admitted):
        """One request on a context of its own, built and freed here (cache off)."""
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

    def _context(self, req0, stream):
        """The scatterer's resident context, built on first use with room for
        merge_rhs right-hand sides; returns (ctx, footprint, built)."""
        key = scatterer_key(req0)
        with self.lock:
            ent = self.contexts[key]
        if ent["ctx"] is None:
            ctx = aim_setup(req0.verts, req0.tris, req0.k, req0.h, M=req0.M, near_radius=req0.near_radius,
                            precision=self.precision, max_rhs=max(self.merge_rhs, len(req0.khat)),
                            stream=stream.cuda_stream, cfie_alpha=req0.cfie_alpha)
            with self.lock:
                ent["ctx"] = ctx
                self.setups += 1
            return ctx, ent["fp"], True
        aim_set_stream(ent["ctx"], stream)
        return ent["ctx"], ent["fp"], False

    def _run_packed(self, groups, stream, admitted):
        """Several scatterers' groups of requests in one multi-instance pack: one
        launch per product stage for all of them (aim_pack_solve).  A pack the
        library refuses (grid layouts that differ after setup) is solved group
        by group instead."""
        torch = self.torch
        nreq = sum(len(grp) for grp in groups)
        try:
            with torch.cuda.stream(stream):
                ctxs, fps, builts = [], [], []
                for grp in groups:
                    ctx, fp, built = self._context(grp[0], stream)
                    ctxs.append(ctx)
                    fps.append(fp)
                    builts.append(built)
                try:
                    pack = aim_pack_create(ctxs, [sum(len(r.khat) for r in grp) for grp in groups])
                except AIMError:
                    return [res for grp in groups for res in self._run_merged(grp, stream, admitted)]
                try:
                    Vs = [aim_rhs_planewave(ctx, np.concatenate([r.khat for r in grp]),
                                            np.concatenate([r.pol for r in grp])) for ctx, grp in zip(ctxs, groups)]
                    X, info = aim_pack_solve(pack, pack.pack(Vs), groups[0][0].tol, raise_on_noconv=False)
                    parts = pack.unpack(X)
                    with self.lock:
                        self.packs.append(len(groups))
                    out = []
                    for i, grp in enumerate(groups):
                        Xi = parts[i]
                        Xh = Xi.cpu().numpy()
                        r0, b0 = pack.b0[i], 0
                        for r in grp:
                            nb = len(r.khat)
                            sigma = None
                            if r.rcs_dirs is not None:
                                sigma = aim_rcs(ctxs[i], Xi[b0 : b0 + nb].contiguous(), *r.rcs_dirs)[0]
                            out.append(Result(r.rid, Xh[b0 : b0 + nb], info["rel_res"][r0 + b0 : r0 + b0 + nb],
                                              info["iterations"], r.arrival, admitted, time.perf_counter() - self.t0,
                                              fps[i], sigma, batch=nreq, setup=builts[i] and r is grp[0]))
                            b0 += nb
                    return out
                finally:
                    pack.close()
        except Exception as e:  # reported per request; the server keeps running
            now = time.perf_counter() - self.t0
            return [Result(r.rid, None, None, 0, r.arrival, admitted, now, 0, error=repr(e), batch=nreq)
                    for grp in groups for r in grp]

    def _run_merged(self, batch, stream, admitted):
        """The batch's right-hand sides in one solve on the scatterer's resident
        context (built here on first use, with room for merge_rhs right-hand sides)."""
        torch = self.torch
        req0 = batch[0]
        fp = 0
        built = False
        try:
            with torch.cuda.stream(stream):
                ctx, fp, built = self._context(req0, stream)
                kh = np.concatenate([r.khat for r in batch])
                po = np.concatenate([r.pol for r in batch])
                V = aim_rhs_planewave(ctx, kh, po)
                X, info = aim_solve(ctx, V, req0.tol, raise_on_noconv=False)
                Xh = X.cpu().numpy()
                out, b0 = [], 0
                for r in batch:
                    nb = len(r.khat)
                    sigma = None
                    if r.rcs_dirs is not None:
                        sigma = aim_rcs(ctx, X[b0 : b0 + nb].contiguous(), *r.rcs_dirs)[0]
                    out.append(Result(r.rid, Xh[b0 : b0 + nb], info["rel_res"][b0 : b0 + nb], info["iterations"],
                                      r.arrival, admitted, time.perf_counter() - self.t0, fp, sigma,
                                      batch=len(batch), setup=built and r is req0))
                    b0 += nb
                return out
        except Exception as e:  # reported per request; the server keeps running
            now = time.perf_counter() - self.t0
            return [Result(r.rid, None, None, 0, r.arrival, admitted, now, fp, error=repr(e), batch=len(batch))
                    for r in batch]

    def _footprint(self, req):
        nrhs = max(self.merge_rhs, len(req.khat)) if self.cache else len(req.khat)
        return aim_footprint(req.verts, req.tris, req.h, req.M, req.near_radius, nrhs, req.cfie_alpha,
                             self.precision)

    def close(self):
        """Free every resident context."""
        with self.lock:
            for ent in self.contexts.values():
                if ent["ctx"] is not None:
                    ent["ctx"].close()
            self.contexts.clear()
            self.claimed = 0

    # -------------------------------------------------------------- driver
    def run(self, requests, realtime=True):
        """Feed requests at their arrival times (or all at once) and wait for all results."""
        self.t0 = time.perf_counter()
        self.stop = False
        threads = [threading.Thread(target=self._worker, args=(i,), daemon=True) for i in range(self.slots)]
        for t in threads:
            t.start()
        for req in sorted(requests, key=lambda r: r.arrival):
            if realtime:
                dt = req.arrival - (time.perf_counter() - self.t0)
                if dt > 0:
                    time.sleep(dt)
            fp = self._footprint(req)
            key = scatterer_key(req) if self.cache else None
            with self.lock:
                self.pending.append((req, fp, key))
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
        "mean_batch": float(np.mean([r.batch for r in ok])) if ok else None,
        "setups": int(sum(1 for r in ok if r.setup)),
    }


def make_stream(n_requests, rate, seed=1, plate_sides=(2, 4, 8, 16, 32), sphere_radii=(1, 2, 4, 8), max_rhs=16,
                theta_max_deg=80.0, sphere_cfie_alpha=1.0, size_jitter=0.0):
    """Synthetic request stream: Poisson arrivals at ``rate`` per second.

    Draw order per request: inter-arrival time, kind (plate or sphere, 50/50),
    size, number of right-hand sides (uniform 1..max_rhs), then the incidence
    angles and polarisations (``aim_inputs.random_incidence``).  Spheres are
    solved with CFIE when ``sphere_cfie_alpha`` < 1 (Section 2.2 uses 0.6 for
    closed bodies); plates are open and always take the EFIE.  With
    ``size_jitter`` > 0 each size is scaled by a factor drawn uniformly from
    [1 - size_jitter, 1 + size_jitter] (after the number of right-hand sides)
    and rounded to 0.01, so nearly every request is a scatterer of its own.
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
        if size_jitter > 0:
            size = round(size * float(rng.uniform(1.0 - size_jitter, 1.0 + size_jitter)), 2)
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
