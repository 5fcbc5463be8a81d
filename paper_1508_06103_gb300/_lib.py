"""ctypes loader of libstkkt.so (the C ABI declared in include/stkkt.h).

Argument marshalling only: every computation happens in the CUDA library.
Loading fails loudly when the library has not been built; there is no
fallback implementation.
"""

from __future__ import annotations

import ctypes as C
import os

from . import build as _build

KKT_OK = 0
KKT_NOT_CONVERGED = 1
KKT_BREAKDOWN = 2
STATUS_NAMES = {0: "OK", 1: "NOT_CONVERGED", 2: "BREAKDOWN", -1: "ERR_ARG", -2: "ERR_NOMEM", -3: "ERR_CUDA",
                -4: "ERR_NONFINITE", -5: "ERR_ZERO_PIVOT"}


class KktGrid(C.Structure):
    _fields_ = [("cx", C.c_int), ("cy", C.c_int), ("cz", C.c_int), ("lx", C.c_double), ("ly", C.c_double),
                ("lz", C.c_double), ("dirichlet_faces", C.c_uint)]


# name: (restype, argtypes) exactly as declared in include/stkkt.h
SIGNATURES = {
    "kkt_last_error": (C.c_char_p, []),
    "kkt_version": (C.c_char_p, []),
    "kkt_create": (C.c_int, [C.POINTER(KktGrid), C.c_int, C.c_double, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int,
                             C.c_double, C.c_double, C.c_double, C.POINTER(C.c_void_p)]),
    "kkt_sizes": (C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int),
                            C.POINTER(C.c_int), C.POINTER(C.c_longlong)]),
    "kkt_rhs": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "kkt_set_regularization": (C.c_int, [C.c_void_p, C.c_int]),
    "kkt_set_element": (C.c_int, [C.c_void_p, C.c_int]),
    "ras_local_pattern": (C.c_int, [C.c_int, C.c_void_p]),
    "kkt_apply": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    "kkt_residual": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "ras_setup": (C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.c_int, C.c_int, C.c_int, C.POINTER(C.c_void_p)]),
    "ras_apply": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "ras_apply_static": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "coarse_setup": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_int), C.c_int,
                               C.c_double, C.c_int, C.c_int, C.POINTER(C.c_void_p)]),
    "two_level_apply": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "reduced_solve": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_double, C.c_int,
                                C.c_double, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "gmres_solve": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_double,
                              C.c_int, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_double), C.c_void_p]),
    "recover_source": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "ras_refactor": (C.c_int, [C.c_void_p, C.c_void_p]),
    "ras_info": (C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_longlong), C.POINTER(C.c_longlong),
                           C.POINTER(C.c_int)]),
    "ras_setup_shape": (C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.c_int, C.c_int, C.c_int, C.POINTER(C.c_int),
                                  C.POINTER(C.c_void_p)]),
    "ras_solve_shape": (C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int),
                                  C.POINTER(C.c_int)]),
    "ras_status": (C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.c_void_p]),
    "ras_setup_batch": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.POINTER(C.c_int), C.c_int, C.c_int,
                                  C.POINTER(C.c_int), C.POINTER(C.c_void_p)]),
    "ras_autotune": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.POINTER(C.c_int), C.c_int, C.c_int, C.c_int,
                               C.c_char_p, C.POINTER(C.c_int), C.POINTER(C.c_double)]),
    "gmres_solve_batch": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int,
                                    C.c_double, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_double),
                                    C.POINTER(C.c_int), C.c_void_p]),
    "ras_selftest_wait": (C.c_int, [C.c_void_p, C.c_double, C.c_void_p]),
    "coarse_refactor": (C.c_int, [C.c_void_p, C.c_void_p]),
    "two_level_refactor": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "kkt_launch_count": (C.c_longlong, []),
    "kkt_fma_peak": (C.c_int, [C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_void_p]),
    "kkt_mma_peak": (C.c_int, [C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_void_p]),
    "kkt_timing_enable": (C.c_int, [C.c_int]),
    "kkt_timing_read": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_longlong)]),
    "ras_timing_read": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_longlong)]),
    "kkt_timing_reset": (C.c_int, [C.c_void_p, C.c_void_p]),
    "kkt_destroy": (None, [C.c_void_p]),
    "ras_destroy": (None, [C.c_void_p]),
    "coarse_destroy": (None, [C.c_void_p]),
}

_LIB = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False) -> C.CDLL:
    """Load the library (optionally building it first); raise if it is absent."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = lib_path()
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"libstkkt.so is not built ({path}); run __graft_entry__.build() "
                               "or python -m paper_1508_06103_gb300.build")
        _build.build()
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


class KktError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def check(status: int, where: str) -> int:
    if status < 0:
        raise KktError(status, where, load().kkt_last_error().decode(errors="replace"))
    return status
