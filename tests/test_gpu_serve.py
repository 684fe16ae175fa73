"""Continuous batching on the GPU: requests of different sizes and
right-hand-side counts run concurrently (one CUDA stream per slot), and each
result equals the same request solved alone (same tolerance gate: true
relative residual <= 1e-6; solutions agree to 1e-10 since every kernel is
deterministic for a given launch shape)."""

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
    s = serve.Server(slots=3)
    # all requests queued at once, so the three slots fill and their work overlaps
    # (with staggered arrivals these small solves can finish before the next arrives)
    mixed, span = s.run(reqs, realtime=False)
    summ = serve.summarize(mixed, span)
    assert summ["failed"] == 0, [r.error for r in mixed]
    assert summ["max_rel_res"] <= 1e-6
    assert s.peak_busy >= 2  # requests overlapped on the device
    for r in reqs:
        alone, _ = serve.Server(slots=1).run([r], realtime=False)
        a, m = alone[0].X, mixed[r.rid].X
        assert np.linalg.norm(a - m) <= 1e-10 * np.linalg.norm(a)


def test_oversubscribed_budget_serialises_but_completes():
    reqs = requests()[:3]
    s = serve.Server(slots=3, mem_budget=1)  # nothing fits: one request at a time
    res, span = s.run(reqs, realtime=False)
    assert all(r.error is None for r in res)
    assert s.peak_busy == 1
