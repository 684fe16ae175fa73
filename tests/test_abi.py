"""The C-ABI library loads and exports every symbol include/aim.h declares (CPU only)."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "aim.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = set(re.findall(r"\b(aim_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_1010_1456_gb300 import _lib

    if not os.path.exists(_lib.LIB_PATH):
        from paper_1010_1456_gb300 import build

        build.build()
    return _lib.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("aim_setup", "aim_matvec", "aim_solve", "aim_rcs", "aim_destroy", "aim_rhs_planewave"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    from paper_1010_1456_gb300 import _lib

    for name in declared_functions():
        assert hasattr(lib, name), name
        assert name in _lib.SIGNATURES, f"binding lacks {name}"


def test_binding_has_no_extra_symbols():
    from paper_1010_1456_gb300 import _lib

    assert set(_lib.SIGNATURES) == set(declared_functions())


def test_error_strings_and_defaults(lib):
    from paper_1010_1456_gb300 import _lib

    assert lib.aim_strerror(_lib.AIM_OK) == b"ok"
    assert lib.aim_strerror(_lib.AIM_ENOCONV) == b"solver did not converge"
    assert lib.aim_strerror(999) == b"unknown error"
    o = _lib.aim_opts()
    lib.aim_default_opts(ctypes.byref(o))
    assert (o.precision, o.restart, o.max_rhs) == (_lib.AIM_C128, 50, 1)
    assert (o.planar, o.cfie_alpha) == (1, 1.0)  # plane collapse on, plain EFIE


def test_null_and_bad_arguments_are_rejected_without_a_device(lib):
    from paper_1010_1456_gb300 import _lib

    h = ctypes.c_void_p()
    # bad scalar arguments fail before any device work
    assert lib.aim_setup(None, 2.0, 0.1, 2, 0.3, None, ctypes.byref(h)) != _lib.AIM_OK
    m = _lib.aim_mesh(0, 0, None, None)
    assert lib.aim_setup(ctypes.byref(m), -1.0, 0.1, 2, 0.3, None, ctypes.byref(h)) == _lib.AIM_EINVAL
    assert lib.aim_setup(ctypes.byref(m), 6.28, 0.1, 7, 0.3, None, ctypes.byref(h)) == _lib.AIM_EINVAL
    assert lib.aim_matvec(None, None, None, 1, _lib.AIM_C128) == _lib.AIM_EINVAL
    assert lib.aim_solve(None, None, None, 1, 1e-6, None) == _lib.AIM_EINVAL
    assert b"null" in lib.aim_last_error()
    assert lib.aim_probe_fma_peak(16, ctypes.byref(ctypes.c_double())) == _lib.AIM_EINVAL
    get = (ctypes.c_int32 * 5)()
    assert lib.aim_fft_config(None, _lib.AIM_C128, None, get) == _lib.AIM_EINVAL
    assert lib.aim_autotune(None, _lib.AIM_C128, 1, 1, None, None) == _lib.AIM_EINVAL
    assert lib.aim_export(None, _lib.AIM_EXPORT_WEIGHTS, None, 0) == _lib.AIM_EINVAL


def test_setup_reports_missing_device(lib):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import numpy as np

    from paper_1010_1456_gb300 import _lib
    from aim_inputs import plate_mesh

    v, t = plate_mesh(1.0, 3)
    v = np.ascontiguousarray(v)
    t = np.ascontiguousarray(t, dtype=np.int32)
    m = _lib.aim_mesh(len(v), len(t), v.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                      t.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    h = ctypes.c_void_p()
    assert lib.aim_setup(ctypes.byref(m), 6.28, 0.1, 2, 0.3, None, ctypes.byref(h)) == _lib.AIM_ENODEV
    assert not h.value


def test_footprint_is_host_only(lib):
    from paper_1010_1456_gb300 import _lib, aim_footprint
    from aim_inputs import icosphere_mesh

    v, t = icosphere_mesh(1.0, 8)
    b1 = aim_footprint(v, t, 0.1, 2, 0.3, 1)
    b8 = aim_footprint(v, t, 0.1, 2, 0.3, 8)
    assert 0 < b1 < b8
    assert aim_footprint(v, t, 0.1, 2, 0.3, 1, cfie_alpha=0.6) > b1
    for bad in (0.0, -0.5, 1.5):  # CFIE weights outside (0, 1]
        with pytest.raises(RuntimeError):
            aim_footprint(v, t, 0.1, 2, 0.3, 1, cfie_alpha=bad)
    # the complex64 solver also holds the float-float refinement grids; native FP64 holds no float-float arrays
    c64 = aim_footprint(v, t, 0.1, 2, 0.3, 4, precision=_lib.AIM_C64)
    c128 = aim_footprint(v, t, 0.1, 2, 0.3, 4, precision=_lib.AIM_C128)
    f64 = aim_footprint(v, t, 0.1, 2, 0.3, 4, precision=_lib.AIM_C128_F64)
    assert c64 > c128 > f64 > 0
    with pytest.raises(RuntimeError):
        aim_footprint(v, t, 0.1, 2, 0.3, 1, precision=7)


def test_non_finite_vertices_and_budget_are_rejected_on_the_host(lib):
    """NaN or infinite coordinates, and a footprint above opts.mem_budget, fail
    before any device work (so also without a GPU)."""
    import numpy as np

    import paper_1010_1456_gb300 as g
    from aim_inputs import plate_mesh
    from paper_1010_1456_gb300 import _lib

    v, t = plate_mesh(1.0, 9)
    for bad in (np.nan, np.inf):
        vb = v.copy()
        vb[3, 1] = bad
        with pytest.raises(g.AIMError) as e:
            g.aim_setup(vb, t, 6.28, 0.1, stream=0)
        assert e.value.code == _lib.AIM_EINVAL
        with pytest.raises(g.AIMError):
            g.aim_footprint(vb, t, 0.1)
    with pytest.raises(g.AIMError) as e:
        g.aim_setup(v, t, 6.28, 0.1, mem_budget=1000, stream=0)
    assert e.value.code == _lib.AIM_ENOMEM
    assert b"mem_budget" in lib.aim_last_error()


def test_pack_arguments_are_checked_on_the_host(lib):
    """aim_pack_* reject null or out-of-range arguments before touching a device."""
    import ctypes as C

    from paper_1010_1456_gb300 import _lib

    out = C.c_void_p()
    nr = (C.c_int32 * 1)(1)
    hs = (C.c_void_p * 1)(None)
    assert lib.aim_pack_create(None, 1, nr, C.byref(out)) == _lib.AIM_EINVAL
    assert lib.aim_pack_create(hs, 0, nr, C.byref(out)) == _lib.AIM_EINVAL
    assert lib.aim_pack_create(hs, 1, nr, C.byref(out)) == _lib.AIM_EINVAL  # a null context
    assert lib.aim_pack_create(hs, 257, nr, C.byref(out)) == _lib.AIM_EINVAL
    assert lib.aim_pack_dims(None, None, None, None) == _lib.AIM_EINVAL
    assert lib.aim_pack_matvec(None, None, None, _lib.AIM_C64) == _lib.AIM_EINVAL
    assert lib.aim_pack_solve(None, None, None, 1e-6, None) == _lib.AIM_EINVAL
    assert lib.aim_pack_set_stream(None, None) == _lib.AIM_EINVAL
    lib.aim_pack_destroy(None)  # a no-op


def test_unknown_krylov_method_is_rejected_on_the_host(lib):
    import paper_1010_1456_gb300 as g
    from aim_inputs import plate_mesh
    from paper_1010_1456_gb300 import _lib

    v, t = plate_mesh(1.0, 9)
    with pytest.raises(g.AIMError) as e:
        g.aim_setup(v, t, 6.28, 0.1, krylov=5, stream=0)
    assert e.value.code == _lib.AIM_EINVAL
    assert lib.aim_set_krylov(None, 0) == _lib.AIM_EINVAL
