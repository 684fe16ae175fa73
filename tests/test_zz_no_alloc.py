"""The complex64 product that allocates nothing (aim_matvec_c64_noalloc).

Some callers cannot let the library call cudaMalloc: their device memory
belongs to another allocator or a fixed pool, or an allocation (which can
synchronise the device) must not happen in their loop.  This entry point
runs the complex64 product on a fixed device array compiled into the
library.  Called through the C ABI, twice in a row on the same inputs, its
result must match aim_matvec with AIM_C64 within the complex64 tolerance used
by the other tests (1e-5 relative), on a plate on the full grid, a plate on
the collapsed planar grid (no z passes), a batch of 3 in a context sized for
4, and an EFIE sphere (whose result is also checked against the oracle).  The
first call on a device is its set-up (the driver maps the fixed array then);
free device memory must not change on the calls after it.  A problem whose
grids exceed the fixed scratch, a batch beyond the context's size, and a call
with another device current are rejected.
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


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _check_twice(ctx, nrhs, seed):
    """Two no-alloc calls in a row equal aim_matvec (AIM_C64); the second takes no memory."""
    x = torch.from_numpy(random_complex((nrhs, ctx.N), seed).astype(np.complex64)).cuda()
    ref = g.aim_matvec(ctx, x, precision=g.AIM_C64).cpu().numpy()
    torch.cuda.synchronize()
    outs = []
    for call in range(2):
        y = torch.full_like(x, complex(np.nan, np.nan))
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        assert _noalloc(ctx, x, y, nrhs) == _lib.AIM_OK, _lib.load().aim_last_error()
        torch.cuda.synchronize()
        if call > 0:  # after the set-up call nothing more is mapped or allocated
            assert torch.cuda.mem_get_info()[0] == free0
        outs.append(y.cpu().numpy())
    for y in outs:
        assert _rel(y, ref) <= 1e-5
    return x, outs[-1]


def test_noalloc_matches_allocating_product_twice():
    v, t = plate_mesh(1.0, 9)
    ctx = g.aim_setup(v, t, K0, H, max_rhs=2, precision=g.AIM_C64, planar=False)
    x, _ = _check_twice(ctx, 2, 31)
    # a third call after the two checked ones, on one RHS: still no device memory taken
    y = torch.empty_like(x)
    free0 = torch.cuda.mem_get_info()[0]
    assert _noalloc(ctx, x, y, 1) == _lib.AIM_OK
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    ctx.close()


def test_noalloc_planar_grid():
    """The plate on its collapsed z = 0 grid (one plane, no z passes)."""
    v, t = plate_mesh(1.0, 9)
    ctx = g.aim_setup(v, t, K0, H, max_rhs=2, precision=g.AIM_C64)
    n, L, _ = g.aim_grid_info(ctx)
    assert n[2] == 1 and L[2] == 1
    _check_twice(ctx, 2, 32)
    ctx.close()


def test_noalloc_partial_batch():
    """A context sized for four right-hand sides called with three."""
    v, t = plate_mesh(1.0, 9)
    ctx = g.aim_setup(v, t, K0, H, max_rhs=4, precision=g.AIM_C64, planar=False)
    _check_twice(ctx, 3, 33)
    ctx.close()


def test_noalloc_efie_sphere_matches_oracle():
    """An EFIE sphere (z passes, group projection in aim_matvec, every group here)."""
    from oracle import aim as oaim
    from oracle.rwg import RWG

    R = 0.5
    v, t = icosphere_mesh(R, icosphere_frequency(R))
    ctx = g.aim_setup(v, t, K0, H, max_rhs=2, precision=g.AIM_C64)
    x, y = _check_twice(ctx, 2, 34)
    op = oaim.AIMOperator(RWG(v, t), K0, H, 2)
    ref = op.matvec(x.cpu().numpy().astype(np.complex128))
    assert _rel(y, ref) <= 1e-5
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


def test_noalloc_rejects_another_current_device():
    """Only where a second GPU is visible: the context's device must be current."""
    if torch.cuda.device_count() < 2:
        pytest.skip("one GPU visible")
    v, t = plate_mesh(1.0, 9)
    ctx = g.aim_setup(v, t, K0, H, max_rhs=1, precision=g.AIM_C64)
    x = torch.zeros((1, ctx.N), dtype=torch.complex64, device="cuda:0")
    y = torch.zeros_like(x)
    with torch.cuda.device(1):
        assert _noalloc(ctx, x, y, 1) == _lib.AIM_EINVAL
    assert b"current" in _lib.load().aim_last_error()
    ctx.close()
