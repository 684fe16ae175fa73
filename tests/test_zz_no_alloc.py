"""The complex64 product that allocates nothing (aim_matvec_c64_noalloc).

It exists for callers that cannot let the library call cudaMalloc (memory
owned by another allocator, or loops where an allocation must not happen).
Called through the C ABI, twice in a row on the same inputs, its result must
match aim_matvec with AIM_C64 within the complex64 tolerance used by the
other tests (1e-5 relative).  The first call on a device is its set-up (the
driver maps the fixed array then); free device memory must not change on
the calls after it.  A problem whose grids exceed the fixed scratch must be
rejected.
"""

import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from aim_inputs import icosphere_frequency, icosphere_mesh, plate_mesh, random_complex  # noqa: E402

import paper_1010_1456_gb300 as g  # noqa: E402
from paper_1010_1456_gb300 import _lib  # noqa: E402

K0, H = 2 * np.pi, 0.1


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


def _noalloc(ctx, x, y, nrhs):
    return _lib.load().aim_matvec_c64_noalloc(ctx.handle, ctypes.c_void_p(x.data_ptr()),
                                              ctypes.c_void_p(y.data_ptr()), nrhs)


def test_noalloc_matches_allocating_product_twice():
    v, t = plate_mesh(1.0, 9)
    ctx = g.aim_setup(v, t, K0, H, max_rhs=2, precision=g.AIM_C64)
    x = torch.from_numpy(random_complex((2, ctx.N), 31).astype(np.complex64)).cuda()
    ref = g.aim_matvec(ctx, x, precision=g.AIM_C64)
    torch.cuda.synchronize()
    outs = []
    for call in range(2):
        y = torch.full_like(x, complex(np.nan, np.nan))
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        assert _noalloc(ctx, x, y, 2) == _lib.AIM_OK, _lib.load().aim_last_error()
        torch.cuda.synchronize()
        if call > 0:  # after the set-up call nothing more is mapped or allocated
            assert torch.cuda.mem_get_info()[0] == free0
        outs.append(y.cpu().numpy())
    # a third call after the two checked ones: still no device memory taken
    free0 = torch.cuda.mem_get_info()[0]
    assert _noalloc(ctx, x, y, 1) == _lib.AIM_OK
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    r = ref.cpu().numpy()
    for y in outs:
        assert np.linalg.norm(y - r) <= 1e-5 * np.linalg.norm(r)
    ctx.close()


def test_noalloc_rejects_grids_beyond_the_scratch():
    R = 4.0
    v, t = icosphere_mesh(R, icosphere_frequency(R))
    ctx = g.aim_setup(v, t, K0, H, max_rhs=1, precision=g.AIM_C64)
    x = torch.zeros((1, ctx.N), dtype=torch.complex64, device="cuda")
    y = torch.zeros_like(x)
    assert _noalloc(ctx, x, y, 1) == _lib.AIM_EINVAL
    assert b"scratch" in _lib.load().aim_last_error()
    assert _noalloc(ctx, x, y, 2) == _lib.AIM_EINVAL  # nrhs beyond max_rhs
    ctx.close()
