"""Continuous batching on the GPU: requests of different sizes and
right-hand-side counts run concurrently (one CUDA stream per slot), and each
result equals the same request solved alone.  Without resident contexts every
request has its own context and launch shapes, so the solutions agree to
1e-10 (every kernel is deterministic for a given launch shape).  With
resident contexts and merged solves a request's right-hand sides share the
launches of the others on its scatterer; each keeps its own Arnoldi process,
but the batch iterates until its last member converges, so the solutions
agree to the solver tolerance: both true relative residuals <= 1e-6 and the
difference within 1e-4 of the solution."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from aim_inputs import icosphere_frequency, icosphere_mesh, plate_mesh, random_incidence  # noqa: E402

import paper_1010_1456_gb300 as g  # noqa: E402
from paper_1010_1456_gb300 import serve  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


def requests():
    meshes = [plate_mesh(1.0, 9), icosphere_mesh(0.5, icosphere_frequency(0.5)), plate_mesh(2.0, 18),
              icosphere_mesh(0.4, icosphere_frequency(0.4))]
    rng = np.random.default_rng(5)
    out = []
    for i, (v, t) in enumerate(meshes + meshes[:2]):
        nrhs = int(rng.integers(1, 5))
        kh, po = random_incidence((nrhs + 1) // 2, rng=rng)
        out.append(serve.Request(i, v, t, kh[:nrhs], po[:nrhs], arrival=0.05 * i))
    return out


def test_results_alone_equal_results_in_the_mix():
    reqs = requests()
    s = serve.Server(slots=3, cache=False)
    # all requests queued at once, so the three slots fill and their work overlaps
    # (with staggered arrivals these small solves can finish before the next arrives)
    mixed, span = s.run(reqs, realtime=False)
    summ = serve.summarize(mixed, span)
    assert summ["failed"] == 0, [r.error for r in mixed]
    assert summ["max_rel_res"] <= 1e-6
    assert s.peak_busy >= 2  # requests overlapped on the device
    for r in reqs:
        alone, _ = serve.Server(slots=1, cache=False).run([r], realtime=False)
        a, m = alone[0].X, mixed[r.rid].X
        assert np.linalg.norm(a - m) <= 1e-10 * np.linalg.norm(a)


def test_oversubscribed_budget_serialises_but_completes():
    reqs = requests()[:3]
    s = serve.Server(slots=3, mem_budget=1, cache=False)  # nothing fits: one request at a time
    res, span = s.run(reqs, realtime=False)
    assert all(r.error is None for r in res)
    assert s.peak_busy == 1


def _true_residual(req, X):
    """||V - Z X|| / ||V|| with the FP64-accurate product on a fresh context."""
    ctx = g.aim_setup(req.verts, req.tris, req.k, req.h, M=req.M, near_radius=req.near_radius,
                      max_rhs=len(req.khat), cfie_alpha=req.cfie_alpha)
    V = g.aim_rhs_planewave(ctx, req.khat, req.pol)
    ZX = g.aim_matvec(ctx, torch.from_numpy(X).cuda(), precision=g.AIM_C128)
    r = (torch.linalg.norm(V - ZX, dim=1) / torch.linalg.norm(V, dim=1)).max().item()
    ctx.close()
    return r


def test_resident_contexts_and_merged_solves_match_alone():
    """Seven requests on three scatterers (a plate and two CFIE spheres), all
    queued at once on two slots: same-scatterer requests merge into one solve
    and reuse the scatterer's resident context, so fewer contexts are built than
    requests; every result meets the tolerance and matches its solve alone."""
    plate = plate_mesh(1.0, 9)
    s05 = icosphere_mesh(0.5, icosphere_frequency(0.5))
    s04 = icosphere_mesh(0.4, icosphere_frequency(0.4))
    rng = np.random.default_rng(9)
    reqs = []
    for i, (v, t), alpha in ((0, plate, 1.0), (1, s05, 0.6), (2, plate, 1.0), (3, s04, 0.6), (4, s05, 0.6),
                             (5, plate, 1.0), (6, s05, 0.6)):
        nrhs = int(rng.integers(1, 5))
        kh, po = random_incidence((nrhs + 1) // 2, rng=rng)
        reqs.append(serve.Request(i, v, t, kh[:nrhs], po[:nrhs], cfie_alpha=alpha))
    s = serve.Server(slots=2, merge_rhs=16)
    res, span = s.run(reqs, realtime=False)
    summ = serve.summarize(res, span)
    assert summ["failed"] == 0, [r.error for r in res]
    assert s.setups == 3 and summ["setups"] == 3  # one context per scatterer
    assert max(s.batches) >= 2  # some solve carried several requests
    for r in reqs:
        m = res[r.rid]
        assert m.rel_res.max() <= 1e-6
        alone, _ = serve.Server(slots=1, cache=False).run([r], realtime=False)
        a = alone[0].X
        assert np.linalg.norm(a - m.X) <= 1e-4 * np.linalg.norm(a), r.rid
        assert _true_residual(r, m.X) <= 1.01e-6
    s.close()


def test_packed_solves_of_different_scatterers_match_alone():
    """Five scatterers of two pack classes (three flat plates, two CFIE spheres),
    all queued at once on one slot with packs of up to four: the plates share a
    pack, the spheres another; every result meets the tolerance and matches its
    solve alone."""
    meshes = [(plate_mesh(1.0, 9), 1.0), (plate_mesh(1.1, 10), 1.0), (icosphere_mesh(0.4, icosphere_frequency(0.4)), 0.6),
              (plate_mesh(0.9, 8), 1.0), (icosphere_mesh(0.45, icosphere_frequency(0.45)), 0.6)]
    rng = np.random.default_rng(12)
    reqs = []
    for i, ((v, t), alpha) in enumerate(meshes):
        nrhs = int(rng.integers(1, 4))
        kh, po = random_incidence((nrhs + 1) // 2, rng=rng)
        reqs.append(serve.Request(i, v, t, kh[:nrhs], po[:nrhs], cfie_alpha=alpha))
    s = serve.Server(slots=1, pack=4)
    res, span = s.run(reqs, realtime=False)
    summ = serve.summarize(res, span)
    assert summ["failed"] == 0, [r.error for r in res]
    assert s.packs and max(s.packs) >= 2  # some solve carried several scatterers
    for r in reqs:
        m = res[r.rid]
        assert m.rel_res.max() <= 1e-6
        alone, _ = serve.Server(slots=1, cache=False).run([r], realtime=False)
        a = alone[0].X
        assert np.linalg.norm(a - m.X) <= 1e-4 * np.linalg.norm(a), r.rid
        assert _true_residual(r, m.X) <= 1.01e-6
    s.close()
