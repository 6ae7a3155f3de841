"""ctypes binding of libhpx.so (the C ABI declared in include/hpx.h).

Argument marshalling only: every step of every transform runs in the CUDA
kernels of libhpx.  Loading fails loudly if the library has not been built.
"""
from __future__ import annotations

import ctypes
import os

import torch  # noqa: F401  -- loads the CUDA runtime libhpx links against

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "lib", "libhpx.so")

HPX_F64, HPX_F32, HPX_F32_BF16, HPX_F32_BF16X3, HPX_F32_FP16, HPX_F32_FP16X3 = range(6)
HPX_PLAN_LAMBDA_RECOMPUTE, HPX_PLAN_LAMBDA_TABLE, HPX_PLAN_TENSOR_CORES, HPX_PLAN_LAMBDA_HOST = 0, 1, 2, 4
HPX_PLAN_TC_TF32X3, HPX_PLAN_LAMBDA_STREAM = 8, 16
HPX_RING, HPX_NESTED, HPX_FLAT = 0, 1, 2
STATUS = {0: "HPX_OK", 1: "HPX_ERR_INVALID", 2: "HPX_ERR_NOMEM", 3: "HPX_ERR_CUDA",
          4: "HPX_ERR_TIMEOUT", 5: "HPX_ERR_UNSUPPORTED"}

# name -> (restype, argtypes); mirrors include/hpx.h
_P, _I, _U, _I64, _SZ = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint, ctypes.c_int64, ctypes.c_size_t
SIGNATURES = {
    "hpx_nalm": (_I64, [_I, _I]),
    "hpx_plan_create": (_I, [_I, _I, _I, _I, _I, ctypes.POINTER(_P)]),
    "hpx_plan_create_ex": (_I, [_I, _I, _I, _I, _I, _U, ctypes.POINTER(_P)]),
    "hpx_plan_create_ooc": (_I, [_I, _I, _I, _I, _I, _SZ, ctypes.POINTER(_P)]),
    "hpx_plan_create_stream": (_I, [_I, _I, _I, _I, _I, _U, _SZ, ctypes.POINTER(_P)]),
    "hpx_plan_test_withhold_copies": (_I, [_P, _I]),
    "hpx_plan_host_bytes": (_SZ, [_P]),
    "hpx_plan_destroy": (_I, [_P]),
    "hpx_map2alm": (_I, [_P, _P, _P, _P]),
    "hpx_alm2map": (_I, [_P, _P, _P, _P]),
    "hpx_map2alm_adjoint": (_I, [_P, _P, _P, _P]),
    "hpx_alm2map_adjoint": (_I, [_P, _P, _P, _P]),
    "hpx_map2alm_noalloc": (_I, [_P, _P, _P, _P]),
    "hpx_map2alm_n": (_I, [_P, _I, _P, _P, _P]),
    "hpx_alm2map_n": (_I, [_P, _I, _P, _P, _P]),
    "hpx_alm2map_grad": (_I, [_P, _P, _P, _P]),
    "hpx_map2alm_grad": (_I, [_P, _P, _P, _P]),
    "hpx_map2alm_host": (_I, [_P, _P, _P, _P]),
    "hpx_map2alm_iter": (_I, [_P, _P, _P, _I, _P]),
    "hpx_map2alm_host_async": (_I, [_P, _P, _P, _P]),
    "hpx_alm2map_host_async": (_I, [_P, _P, _P, _P]),
    "hpx_plan_host_sync": (_I, [_P]),
    "hpx_alm2map_host": (_I, [_P, _P, _P, _P]),
    "hpx_plan_device_bytes": (_SZ, [_P]),
    "hpx_plan_ring_table": (_I, [_P, _P, _P, _P, _P, _P]),
    "hpx_plan_set_timing": (_I, [_P, _I]),
    "hpx_plan_stage_times": (_I, [_P, _P, _P]),
    "hpx_plan_chain_stats": (_I, [_P, _P, _P]),
    "hpx_plan_table_bytes": (_SZ, [_P]),
    "hpx_plan_column_table_bytes": (_SZ, [_P]),
    "hpx_plan_estimate_bytes": (_SZ, [_I, _I, _I, _I, _I, _U]),
    "hpx_plan_device_status": (_I, [_P]),
    "hpx_plan_set_ring_weights": (_I, [_P, _P, _I]),
    "hpx_reorder": (_I, [_I, _I, _SZ, _I, _I, _P, _P, _P]),
    "hpx_layout_index": (_I, [_I, _I, _I, _P, _P]),
    "hpx_layout_status": (_I, []),
    "hpx_last_error": (ctypes.c_char_p, []),
}

_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"libhpx.so not found at {LIB_PATH}; build it first "
                "(python -c 'import __graft_entry__ as g; g.build()')")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class HpxError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = lib().hpx_last_error().decode(errors="replace")
        super().__init__(f"{where}: {STATUS.get(status, status)}: {msg}")
        self.status = status


def check(status: int, where: str) -> None:
    if status != 0:
        raise HpxError(status, where)
