"""Host-side logic of the request loop (CPU only): admission by footprint,
slot limits, arrival order, failure isolation.  The solve itself is replaced
by a fake that sleeps, so no GPU is touched."""

import threading
import time

import numpy as np
import pytest

from paper_1010_1456_gb300 import serve


class FakeServer(serve.Server):
    def __init__(self, footprints, durations, fail=(), **kw):
        kw.setdefault("cache", False)
        super().__init__(**kw)
        self.fps = footprints
        self.durs = durations
        self.fail = set(fail)
        self.live = 0
        self.live_lock = threading.Lock()
        self.max_live = 0
        self.order = []

    def _make_stream(self):
        return None

    def _footprint(self, req):
        return self.fps[req.rid]

    def _run(self, req, fp, stream, admitted):
        with self.live_lock:
            self.live += 1
            self.max_live = max(self.max_live, self.live)
            self.order.append(req.rid)
        time.sleep(self.durs[req.rid])
        with self.live_lock:
            self.live -= 1
        if req.rid in self.fail:
            return serve.Result(req.rid, None, None, 0, req.arrival, admitted, time.perf_counter() - self.t0, fp,
                                error="injected")
        return serve.Result(req.rid, np.zeros((1, 1)), np.array([0.0]), 1, req.arrival, admitted,
                            time.perf_counter() - self.t0, fp)


def reqs(n, gap=0.0):
    v = np.zeros((3, 3))
    t = np.zeros((1, 3), dtype=np.int32)
    return [serve.Request(i, v, t, np.zeros((1, 3)), np.zeros((1, 3)), arrival=i * gap) for i in range(n)]


def test_budget_and_slots_are_respected():
    fps = [40, 40, 40, 70, 10, 10]
    s = FakeServer(fps, [0.05] * 6, slots=3, mem_budget=100)
    res, span = s.run(reqs(6), realtime=False)
    assert all(r.error is None for r in res)
    assert s.peak_claimed <= 100
    assert s.max_live <= 3
    assert s.peak_busy >= 2  # work overlapped


def test_oversized_request_runs_alone():
    s = FakeServer([500, 10], [0.02, 0.02], slots=2, mem_budget=100)
    res, _ = s.run(reqs(2), realtime=False)
    assert all(r.error is None for r in res)


def test_small_requests_pass_a_blocked_large_one():
    # request 1 does not fit while 0 runs; request 2 does and is admitted first
    fps = [80, 50, 10]
    s = FakeServer(fps, [0.2, 0.01, 0.01], slots=3, mem_budget=100)
    res, _ = s.run(reqs(3), realtime=False)
    assert s.order.index(2) < s.order.index(1)


def test_failure_is_isolated_and_summarised():
    s = FakeServer([1, 1, 1], [0.01] * 3, fail=[1], slots=2, mem_budget=100)
    res, span = s.run(reqs(3), realtime=False)
    summ = serve.summarize(res, span)
    assert summ["solves"] == 2 and summ["failed"] == 1
    assert summ["p50_s"] is not None and summ["p99_s"] >= summ["p50_s"]


def test_poisson_stream_draws_are_seeded():
    a = serve.make_stream(6, rate=2.0, seed=1, plate_sides=(1,), sphere_radii=(0.5,), max_rhs=3)
    b = serve.make_stream(6, rate=2.0, seed=1, plate_sides=(1,), sphere_radii=(0.5,), max_rhs=3)
    assert [r.arrival for r in a] == [r.arrival for r in b]
    assert [r.label for r in a] == [r.label for r in b]
    assert all(1 <= len(r.khat) <= 3 for r in a)
    assert np.all(np.diff([r.arrival for r in a]) > 0)


def test_cfie_is_requested_for_spheres_only():
    """The stream's closed bodies (spheres) take the CFIE alpha; plates are open
    and stay on the EFIE; the draws do not depend on alpha."""
    a = serve.make_stream(12, rate=2.0, seed=3, plate_sides=(1,), sphere_radii=(0.5,), max_rhs=2,
                          sphere_cfie_alpha=0.6)
    b = serve.make_stream(12, rate=2.0, seed=3, plate_sides=(1,), sphere_radii=(0.5,), max_rhs=2)
    assert [r.label for r in a] == [r.label for r in b]
    assert {r.cfie_alpha for r in a if r.label.startswith("plate")} == {1.0}
    assert {r.cfie_alpha for r in a if r.label.startswith("sphere")} == {0.6}
    assert {r.cfie_alpha for r in b} == {1.0}


class FakeMergingServer(serve.Server):
    """Resident contexts and merged solves with the solve replaced by a sleep:
    records which requests each solve took and whether it had to build."""

    def __init__(self, footprints, duration=0.02, **kw):
        super().__init__(**kw)
        self.fps = footprints
        self.duration = duration
        self.solves = []

    def _make_stream(self):
        return None

    def _footprint(self, req):
        return self.fps[req.rid]

    def _run_merged(self, batch, stream, admitted):
        key = serve.scatterer_key(batch[0])
        with self.lock:
            ent = self.contexts[key]
            built = ent["ctx"] is None
            if built:
                ent["ctx"] = _FakeCtx()
                self.setups += 1
        self.solves.append(([r.rid for r in batch], built))
        time.sleep(self.duration)
        now = time.perf_counter() - self.t0
        return [serve.Result(r.rid, np.zeros((len(r.khat), 1)), np.zeros(len(r.khat)), 1, r.arrival, admitted, now,
                             ent["fp"], batch=len(batch), setup=built and r is batch[0]) for r in batch]


class _FakeCtx:
    closed = 0

    def close(self):
        _FakeCtx.closed += 1


def mesh_reqs(kinds, nrhs=1):
    """Requests on scatterers named by `kinds` (equal names share a mesh)."""
    meshes = {}
    out = []
    for i, k in enumerate(kinds):
        if k not in meshes:
            v = np.zeros((3, 3))
            v[0, 0] = float(len(meshes) + 1)  # distinct vertex coordinates per scatterer
            meshes[k] = (v, np.array([[0, 1, 2]], dtype=np.int32))
        v, t = meshes[k]
        out.append(serve.Request(i, v, t, np.zeros((nrhs, 3)), np.zeros((nrhs, 3)), label=k))
    return out


def test_same_scatterer_requests_merge_and_reuse_the_resident_context():
    """Queued requests for one scatterer are solved together; a later request
    for it reuses the resident context instead of building another."""
    reqs = mesh_reqs(["a", "a", "b", "a", "b"], nrhs=2)
    s = FakeMergingServer([10] * 5, slots=1, mem_budget=100, merge_rhs=4)
    res, _ = s.run(reqs, realtime=False)
    assert all(r.error is None for r in res)
    # one slot: the first solve takes a0 with a1 (4 RHS, the merge limit), then b2 with b4, then a3 alone
    assert s.solves == [([0, 1], True), ([2, 4], True), ([3], False)]
    assert s.setups == 2
    summ = serve.summarize(res, 1.0)
    assert summ["setups"] == 2 and summ["mean_batch"] == pytest.approx((2 + 2 + 2 + 2 + 1) / 5)


def test_idle_resident_contexts_are_evicted_for_room():
    """Three scatterers of 40 bytes each under a budget of 100: the third one's
    context needs the least recently used idle one freed."""
    _FakeCtx.closed = 0
    reqs = mesh_reqs(["a", "b", "c"])
    s = FakeMergingServer([40, 40, 40], slots=1, mem_budget=100)
    res, _ = s.run(reqs, realtime=False)
    assert all(r.error is None for r in res)
    assert _FakeCtx.closed == 1 and len(s.contexts) == 2 and s.claimed == 80
    assert s.peak_claimed <= 100
    s.close()
    assert s.claimed == 0 and not s.contexts


def test_busy_context_makes_its_requests_wait_not_duplicate():
    """Two slots, two requests for one scatterer arriving one after the other:
    the second waits for the context (or merges) instead of building a second one."""
    reqs = mesh_reqs(["a", "a"])
    reqs[1].arrival = 0.005
    s = FakeMergingServer([10, 10], duration=0.05, slots=2, mem_budget=100)
    res, _ = s.run(reqs, realtime=True)
    assert all(r.error is None for r in res)
    assert s.setups == 1


class FakePackingServer(serve.Server):
    """Packs with the solves replaced by a sleep: records the scatterers of each solve."""

    def __init__(self, footprints, duration=0.02, **kw):
        super().__init__(**kw)
        self.fps = footprints
        self.duration = duration
        self.solves = []

    def _make_stream(self):
        return None

    def _footprint(self, req):
        return self.fps[req.rid]

    def _finish(self, groups, admitted):
        with self.lock:
            for grp in groups:
                ent = self.contexts[serve.scatterer_key(grp[0])]
                if ent["ctx"] is None:
                    ent["ctx"] = _FakeCtx()
                    self.setups += 1
        self.solves.append([[r.rid for r in grp] for grp in groups])
        time.sleep(self.duration)
        now = time.perf_counter() - self.t0
        n = sum(len(grp) for grp in groups)
        return [serve.Result(r.rid, np.zeros((len(r.khat), 1)), np.zeros(len(r.khat)), 1, r.arrival, admitted, now, 1,
                             batch=n) for grp in groups for r in grp]

    def _run_packed(self, groups, stream, admitted):
        return self._finish(groups, admitted)

    def _run_merged(self, batch, stream, admitted):
        return self._finish([batch], admitted)


def shaped_reqs(shapes, nrhs=1):
    """One request per (name, extent x, extent y, extent z): equal names share a mesh."""
    meshes, out = {}, []
    for i, (name, ex, ey, ez) in enumerate(shapes):
        if name not in meshes:
            v = np.array([[0.0, 0.0, 0.0], [ex, 0.0, 0.0], [0.0, ey, ez]])
            meshes[name] = (v, np.array([[0, 1, 2]], dtype=np.int32))
        v, t = meshes[name]
        out.append(serve.Request(i, v, t, np.zeros((nrhs, 3)), np.zeros((nrhs, 3)), label=name))
    return out


def test_pack_takes_other_scatterers_of_its_class():
    """One slot, pack of up to 3: three flat scatterers of similar size share the
    first solve; the curved one (another grid layout), the much larger flat one
    (box volume beyond the ratio) and the fourth flat one (pack full) wait."""
    reqs = shaped_reqs([("a", 1.0, 1.0, 0.0), ("b", 1.1, 0.9, 0.0), ("s", 0.5, 0.5, 0.5), ("c", 1.2, 1.0, 0.0),
                        ("big", 6.0, 6.0, 0.0), ("d", 1.0, 1.1, 0.0)])
    s = FakePackingServer([10] * 6, slots=1, mem_budget=1000, pack=3, pack_ratio=4.0)
    res, _ = s.run(reqs, realtime=False)
    assert all(r.error is None for r in res)
    assert s.solves[0] == [[0], [1], [3]]
    assert sorted(sum(s.solves[1:], []), key=lambda g: g[0]) == [[2], [4], [5]]
    assert s.setups == 6


def test_pack_respects_budget_and_rhs_limit():
    """A scatterer whose new context would exceed the budget, or whose right-hand
    sides would exceed pack_rhs, is left for a later solve."""
    reqs = shaped_reqs([("a", 1.0, 1.0, 0.0), ("b", 1.01, 1.0, 0.0), ("c", 1.02, 1.0, 0.0),
                        ("d", 1.03, 1.0, 0.0)], nrhs=3)
    s = FakePackingServer([40, 70, 40, 10], slots=1, mem_budget=100, pack=4, pack_rhs=6)
    res, _ = s.run(reqs, realtime=False)
    assert all(r.error is None for r in res)
    # b does not fit beside a (40 + 70 > 100); c does (80), and a + c fill pack_rhs = 6
    assert s.solves[0] == [[0], [2]]
    assert [[1], [3]] in s.solves[1:] or [[1]] in s.solves[1:]
    assert s.peak_claimed <= 100


def test_pack_of_one_scatterer_is_a_merged_solve():
    reqs = shaped_reqs([("a", 1.0, 1.0, 0.0), ("a", 1.0, 1.0, 0.0)])
    s = FakePackingServer([10, 10], slots=1, mem_budget=100, pack=4)
    res, _ = s.run(reqs, realtime=False)
    assert s.solves == [[[0, 1]]]


def test_pack_class_and_box_volume():
    """Flat meshes (constant z) get the planar class and a one-plane box; the
    box grows with the bounding box in grid steps."""
    flat = serve.Request(0, np.array([[0.0, 0, 0], [1.0, 0, 0], [0, 1.0, 0]]), np.zeros((1, 3), np.int32),
                         np.zeros((1, 3)), np.zeros((1, 3)))
    solid = serve.Request(1, np.array([[0.0, 0, 0], [1.0, 0, 0], [0, 1.0, 0.5]]), np.zeros((1, 3), np.int32),
                          np.zeros((1, 3)), np.zeros((1, 3)))
    assert serve.pack_class(flat)[-1] is True and serve.pack_class(solid)[-1] is False
    assert serve.pack_class(flat)[:4] == serve.pack_class(solid)[:4]
    # h = 0.1, M = 2: 10 + 4 nodes per unit side, one plane when flat
    assert serve.box_volume(flat) == 14 * 14 * 1
    assert serve.box_volume(solid) == 14 * 14 * 9


def test_pack_rows_layout_on_the_host():
    """Pack.pack / unpack place instance i's [nrhs_i, N_i] block at rows
    b0_i.. and columns 0..N_i - 1 of the [B, ld] array, zeros elsewhere."""
    torch = pytest.importorskip("torch")
    from paper_1010_1456_gb300 import Pack

    class C:
        def __init__(self, N):
            self.N = N

    p = Pack(None, [C(3), C(5)], [2, 1], 5, 3, [0, 2])
    a = torch.arange(6, dtype=torch.float64).reshape(2, 3) + 1
    b = torch.arange(5, dtype=torch.float64).reshape(1, 5) + 10
    packed = p.pack([a, b])
    assert packed.shape == (3, 5)
    assert torch.equal(packed[:2, :3], a) and torch.count_nonzero(packed[:2, 3:]).item() == 0
    assert torch.equal(packed[2:, :], b)
    ua, ub = p.unpack(packed)
    assert torch.equal(ua, a) and torch.equal(ub, b)
