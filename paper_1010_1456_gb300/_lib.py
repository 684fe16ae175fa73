"""ctypes declarations of the C ABI in include/aim.h (argument marshalling only).

The shared library is the in-tree ``libaim.so`` built by ``build.py``.  If it
is missing, importing the binding raises: there is no fallback.
"""

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
# AIM_LIBRARY selects another build of the library in this tree, e.g. the
# index-checking debug build libaim_check.so (build.py --check)
LIB_PATH = os.path.join(HERE, os.environ.get("AIM_LIBRARY", "libaim.so"))

AIM_OK, AIM_EINVAL, AIM_ENOMEM, AIM_ECUDA, AIM_ENOCONV, AIM_ETIMEOUT, AIM_ENODEV = range(7)
AIM_C64, AIM_C128, AIM_C128_F64 = 1, 2, 3
AIM_GMRES, AIM_TFQMR = 0, 1
(AIM_EXPORT_ANCHORS, AIM_EXPORT_WEIGHTS, AIM_EXPORT_NEAR_PTR, AIM_EXPORT_NEAR_COL, AIM_EXPORT_NEAR_VAL,
 AIM_EXPORT_DIAG, AIM_EXPORT_GHAT, AIM_EXPORT_PROJ_PTR, AIM_EXPORT_MFIE_WEIGHTS) = range(1, 10)


class aim_mesh(C.Structure):
    _fields_ = [("nv", C.c_int32), ("nt", C.c_int32), ("verts", C.POINTER(C.c_double)), ("tris", C.POINTER(C.c_int32))]


class aim_opts(C.Structure):
    _fields_ = [
        ("precision", C.c_int),
        ("restart", C.c_int),
        ("maxit", C.c_int),
        ("check_every", C.c_int),
        ("max_rhs", C.c_int),
        ("verbose", C.c_int),
        ("stream", C.c_void_p),
        ("planar", C.c_int),
        ("cfie_alpha", C.c_double),
        ("mem_budget", C.c_size_t),
        ("krylov", C.c_int),
    ]


class aim_solve_info(C.Structure):
    _fields_ = [
        ("iterations", C.c_int32),
        ("restarts", C.c_int32),
        ("rel_res", C.POINTER(C.c_double)),
        ("converged", C.POINTER(C.c_int32)),
    ]


# name -> (restype, argtypes); mirrors include/aim.h
SIGNATURES = {
    "aim_default_opts": (None, [C.POINTER(aim_opts)]),
    "aim_setup": (C.c_int, [C.POINTER(aim_mesh), C.c_double, C.c_double, C.c_int, C.c_double, C.POINTER(aim_opts),
                            C.POINTER(C.c_void_p)]),
    "aim_destroy": (None, [C.c_void_p]),
    "aim_set_stream": (C.c_int, [C.c_void_p, C.c_void_p]),
    "aim_set_precision": (C.c_int, [C.c_void_p, C.c_int]),
    "aim_set_krylov": (C.c_int, [C.c_void_p, C.c_int]),
    "aim_num_unknowns": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64)]),
    "aim_grid_info": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int64)]),
    "aim_rhs_planewave": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_void_p]),
    "aim_matvec": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int]),
    "aim_matvec_c64_noalloc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]),
    "aim_matvec_host": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int]),
    "aim_solve": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_double, C.POINTER(aim_solve_info)]),
    "aim_rcs": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double),
                          C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "aim_rcs_grid": (C.c_int, [C.c_int, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double),
                               C.POINTER(C.c_double)]),
    "aim_err_thth": (C.c_int, [C.c_int, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double),
                               C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "aim_mie_sigma_thth": (C.c_int, [C.c_double, C.c_double, C.c_int, C.POINTER(C.c_double),
                                     C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "aim_footprint": (C.c_int, [C.POINTER(aim_mesh), C.c_double, C.c_int, C.c_double, C.c_int, C.c_double,
                                C.c_int, C.POINTER(C.c_size_t)]),
    "aim_export": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_size_t]),
    "aim_launch_count": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64)]),
    "aim_profile": (C.c_int, [C.c_void_p, C.c_int]),
    "aim_profile_read": (C.c_int, [C.c_void_p, C.c_int, C.c_char_p, C.POINTER(C.c_int64), C.POINTER(C.c_double),
                                   C.POINTER(C.c_int)]),
    "aim_probe_fma_peak": (C.c_int, [C.c_int, C.POINTER(C.c_double)]),
    "aim_fft_config": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "aim_autotune": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_int32), C.POINTER(C.c_double)]),
    "aim_pack_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.POINTER(C.c_int32), C.POINTER(C.c_void_p)]),
    "aim_pack_dims": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "aim_pack_matvec": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]),
    "aim_pack_solve": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.POINTER(aim_solve_info)]),
    "aim_pack_set_stream": (C.c_int, [C.c_void_p, C.c_void_p]),
    "aim_pack_destroy": (None, [C.c_void_p]),
    "aim_strerror": (C.c_char_p, [C.c_int]),
    "aim_last_error": (C.c_char_p, []),
}

_lib = None


def load():
    """Load libaim.so once and attach the signatures; raise if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"{LIB_PATH} is missing: build the CUDA library first "
            "(python -m paper_1010_1456_gb300.build); there is no CPU fallback"
        )
    lib = C.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class AIMError(RuntimeError):
    def __init__(self, code, where):
        lib = load()
        msg = lib.aim_strerror(code).decode()
        detail = lib.aim_last_error().decode()
        super().__init__(f"{where}: {msg} ({detail})")
        self.code = code


def check(code, where):
    if code != AIM_OK:
        raise AIMError(code, where)
    return code
