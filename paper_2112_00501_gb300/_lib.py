"""ctypes declarations of the C ABI in include/mgc.h.

Argument marshalling only: every computation runs in libmgc.so.  Loading fails
loudly when the library has not been built; there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIBPATH = os.path.join(_HERE, "libmgc.so")

MGC_OK = 0
MGC_ERR_INVALID_ARG = 1
MGC_ERR_UNSUPPORTED_SHAPE = 2
MGC_ERR_NOT_UNITARY = 3
MGC_ERR_CUDA = 4
MGC_NOT_CONVERGED = 5
MGC_ERR_BREAKDOWN = 6
MGC_ERR_TIMEOUT = 7
MGC_ERR_NO_DEVICE = 8


class SolveParams(C.Structure):
    _fields_ = [
        ("method", C.c_int),
        ("precond", C.c_int),
        ("smoother_prec", C.c_int),
        ("n_cy", C.c_int),
        ("n_mr", C.c_int),
        ("restart", C.c_int),
        ("tol", C.c_double),
        ("max_iter", C.c_int),
        ("on_device", C.c_int),
        ("x_is_guess", C.c_int),
        ("inner_tol", C.c_double),
        ("sap_solver", C.c_int),
    ]


class MgParams(C.Structure):
    _fields_ = [
        ("n_cy", C.c_int),
        ("n_jacobi", C.c_int),
        ("smoother_prec", C.c_int),
        ("coarse_tol", C.c_double),
        ("coarse_maxit", C.c_int),
        ("n_adapt", C.c_int),
    ]


class SolveInfo(C.Structure):
    _fields_ = [
        ("status", C.c_int),
        ("iters", C.c_int),
        ("restarts", C.c_int),
        ("true_res", C.c_double),
    ]


# name -> (restype, argtypes)
_P = C.c_void_p
_I = C.c_int
_D = C.c_double
SIGNATURES = {
    "mgc_version": (_I, []),
    "mgc_status_string": (C.c_char_p, [_I]),
    "mgc_last_error": (C.c_char_p, []),
    "mgc_counters": (_I, [C.POINTER(C.c_longlong), C.POINTER(_D), _I]),
    "mgc_lattice_create": (_I, [C.POINTER(_I), C.POINTER(_I), _I, C.POINTER(_P)]),
    "mgc_lattice_destroy": (_I, [_P]),
    "mgc_lattice_volume": (C.c_longlong, [_P]),
    "mgc_spinor_bytes": (C.c_size_t, [_P, _I, _I]),
    "mgc_spinor_pack": (_I, [_P, _I, _I, _P, _P, _P]),
    "mgc_spinor_unpack": (_I, [_P, _I, _I, _P, _P, _P]),
    "mgc_spinor_convert": (_I, [_P, _I, _I, _P, _I, _P, _P]),
    "mgc_gauge_create": (_I, [_P, _P, _I, _I, _I, _P, C.POINTER(_P)]),
    "mgc_gauge_destroy": (_I, [_P]),
    "mgc_clover_create": (_I, [_P, _D, _D, _P, C.POINTER(_P)]),
    "mgc_clover_destroy": (_I, [_P]),
    "mgc_device_status": (_I, [_P, C.POINTER(_I), _I, _P]),
    "mgc_selftest_bounded_wait": (_I, [C.c_longlong, _I, C.POINTER(_I), _P]),
    "mgc_fma_peak": (_I, [_I, C.POINTER(C.c_double), _P]),
    "mgc_clover_export": (_I, [_P, _I, _P, _P]),
    "mgc_apply_D": (_I, [_P, _P, _P, _I, _I, _P]),
    "mgc_apply_Ddag": (_I, [_P, _P, _P, _I, _I, _P]),
    "mgc_apply_clover": (_I, [_P, _P, _P, _I, _I, _I, _P]),
    "mgc_sap_smooth": (_I, [_P, _P, _P, _I, _I, _I, _I, _I, _P]),
    "mgc_apply_A": (_I, [_P, _P, _P, _I, _I, _P]),
    "mgc_sap_smooth_eo": (_I, [_P, _P, _P, _I, _I, _I, _I, _I, _P]),
    "mgc_sap_smooth_A": (_I, [_P, _P, _P, _I, _I, _I, _I, _I, _P]),
    "mgc_solve_params_default": (None, [C.POINTER(SolveParams)]),
    "mgc_solve": (_I, [_P, _P, _P, _I, C.POINTER(SolveParams), C.POINTER(SolveInfo), _P]),
    "mgc_force": (_I, [_P, _P, _P, C.POINTER(SolveParams), C.POINTER(SolveInfo), _P, _P]),
    "mgc_solve_noalloc": (_I, [_P, _P, _P, C.POINTER(SolveParams), C.POINTER(SolveInfo), _P]),
    "mgc_mg_params_default": (None, [C.POINTER(MgParams)]),
    "mgc_mg_create": (_I, [_P, C.POINTER(_I), _I, C.POINTER(_P)]),
    "mgc_mg_destroy": (_I, [_P]),
    "mgc_mg_coarse_volume": (C.c_longlong, [_P]),
    "mgc_mg_setup": (_I, [_P, _P, C.POINTER(MgParams), _P]),
    "mgc_mg_set_vectors": (_I, [_P, _P, _P]),
    "mgc_mg_export": (_I, [_P, _P, _P, _P]),
    "mgc_mg_restrict": (_I, [_P, _P, _P, _P]),
    "mgc_mg_prolong": (_I, [_P, _P, _P, _P]),
    "mgc_mg_coarse_apply": (_I, [_P, _P, _P, _P]),
    "mgc_mg_coarse_solve": (_I, [_P, _P, _P, _D, _I, C.POINTER(_I), _P]),
    "mgc_mg_precond": (_I, [_P, _P, _P, C.POINTER(MgParams), _P]),
    "mgc_mg_solve": (_I, [_P, _P, _P, C.POINTER(SolveParams), C.POINTER(MgParams), C.POINTER(SolveInfo), _P]),
    "mgc_batch_create": (_I, [C.POINTER(_P), C.POINTER(_I), _I, C.POINTER(_P)]),
    "mgc_batch_destroy": (_I, [_P]),
    "mgc_batch_systems": (_I, [_P]),
    "mgc_batch_apply_D": (_I, [_P, C.POINTER(_P), C.POINTER(_P), _I, _I, _P]),
    "mgc_batch_sap_smooth": (_I, [_P, C.POINTER(_P), C.POINTER(_P), _I, _I, _I, _I, _P]),
    "mgc_batch_solve": (_I, [_P, C.POINTER(_P), C.POINTER(_P), C.POINTER(SolveParams), C.POINTER(SolveInfo),
                             _P]),
    "mgc_batch_tune": (_I, [_P, _I, _I, C.POINTER(_I), C.POINTER(_I), C.POINTER(_I), C.POINTER(_I), _P]),
    "mgc_batch_set_shape": (_I, [_P, _I, _I, _I, _I, _I]),
}

MGC_BATCH_MAX = 8

_lib = None


def load() -> C.CDLL:
    """The loaded libmgc.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIBPATH):
            raise ImportError(f"{LIBPATH} is missing: build it with "
                              "`python -m paper_2112_00501_gb300.build`")
        lib = C.CDLL(LIBPATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


class MgcError(RuntimeError):
    def __init__(self, status: int, where: str):
        lib = load()
        msg = lib.mgc_last_error().decode(errors="replace")
        super().__init__(f"{where}: {lib.mgc_status_string(status).decode()} ({status}): {msg}")
        self.status = status


def check(status: int, where: str) -> int:
    if status != MGC_OK:
        raise MgcError(status, where)
    return status
