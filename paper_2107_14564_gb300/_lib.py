"""ctypes view of libbispec.so (the C ABI declared in include/bispec.h).

Argument marshalling only. The library is loaded from this package's directory; if it is
missing, loading raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libbispec.so")

BSP_OK = 0
STATUS_NAMES = {0: "BSP_OK", 1: "BSP_ERR_INVALID_ARG", 2: "BSP_ERR_ALIASING", 3: "BSP_ERR_OOM",
                4: "BSP_ERR_CUDA", 5: "BSP_ERR_TIMEOUT", 6: "BSP_ERR_NOT_SUPPORTED",
                7: "BSP_ERR_NUMERIC"}
PRECISIONS = {"fp64": 0, "fp32": 1, "mixed_bf16x3": 2}


class PlanDesc(C.Structure):
    _fields_ = [("ng", C.c_int), ("box_len", C.c_double), ("n_shells", C.c_int),
                ("edges_kf", C.POINTER(C.c_double)), ("n_mu", C.c_int), ("n_t", C.c_int),
                ("rsd", C.c_int), ("beta", C.c_double), ("precision", C.c_int),
                ("mem_budget_bytes", C.c_size_t), ("autotune", C.c_int),
                ("k1_merge", C.c_int),
                ("label_k", C.c_int),
                ("dim", C.c_int),
                ("order", C.c_int)]


class Triplet(C.Structure):
    _fields_ = [("a", C.c_int), ("b", C.c_int), ("c", C.c_int), ("i_mu", C.c_int), ("i_t", C.c_int),
                ("inside", C.c_int), ("ntri", C.c_double), ("tsum", C.c_double), ("k1", C.c_double),
                ("k2", C.c_double), ("k3", C.c_double), ("mu", C.c_double), ("t", C.c_double),
                ("e", C.c_int), ("reserved", C.c_int)]


class BispecError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


# name -> (restype, argtypes)
SIGNATURES = {
    "bsp_plan_create": (C.c_int, [C.POINTER(PlanDesc), C.c_void_p, C.POINTER(C.c_void_p)]),
    "bsp_plan_destroy": (C.c_int, [C.c_void_p]),
    "bsp_plan_info": (C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                C.POINTER(C.c_size_t), C.POINTER(C.c_size_t)]),
    "bsp_plan_grid": (C.c_int, [C.c_void_p, C.POINTER(C.c_int)]),
    "bsp_plan_host_input_bytes": (C.c_int, [C.c_void_p, C.POINTER(C.c_size_t)]),
    "bsp_plan_slabs": (C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "bsp_plan_pass_tuning": (C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "bsp_plan_tuning": (C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int), C.c_int]),
    "bsp_plan_bin_levels": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "bsp_plan_triplets": (C.c_int, [C.c_void_p, C.POINTER(C.POINTER(Triplet)), C.POINTER(C.c_int)]),
    "bsp_shell_fields": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "bsp_contract": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "bsp_estimate": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "bsp_estimate_host": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "bsp_estimate_batched": (C.c_int, [C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), C.c_int,
                                       C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), C.c_void_p]),
    "bsp_batch_create": (C.c_int, [C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), C.c_int,
                                   C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), C.c_void_p,
                                   C.POINTER(C.c_void_p)]),
    "bsp_batch_run": (C.c_int, [C.c_void_p, C.c_void_p]),
    "bsp_batch_destroy": (C.c_int, [C.c_void_p]),
    "bsp_spectrum": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "bsp_grad": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "bsp_last_sums": (C.c_int, [C.c_void_p, C.POINTER(C.c_void_p)]),
    "bsp_plan_check": (C.c_int, [C.c_void_p, C.c_void_p]),
    "bsp_selftest_wait_timeout": (C.c_int, [C.c_void_p, C.c_void_p]),
    "bsp_timing_enable": (C.c_int, [C.c_void_p, C.c_int, C.c_int]),
    "bsp_timing_read": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int),
                                  C.POINTER(C.c_longlong)]),
    "bsp_plan_stage_work": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "bsp_triple_sums_noalloc": (C.c_int, [C.c_void_p, C.c_int, C.c_longlong, C.c_void_p, C.c_int,
                                          C.c_void_p, C.c_void_p]),
    "bsp_last_error": (C.c_char_p, []),
    "bsp_version": (C.c_char_p, []),
}

_lib = None


def load():
    """Load libbispec.so once (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with "
                          "`python -m paper_2107_14564_gb300.build`")
    lib = C.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(status: int):
    if status != BSP_OK:
        msg = load().bsp_last_error().decode(errors="replace")
        raise BispecError(status, msg)
