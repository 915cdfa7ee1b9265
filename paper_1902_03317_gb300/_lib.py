"""ctypes binding of libpasta (include/pasta.h): argument marshalling only.

Every computation runs in the CUDA library; this module converts Python and
torch objects into the C ABI's plain pointers and sizes.  If the library has
not been built, loading fails with a RuntimeError (there is no CPU fallback).
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libpasta.so")

PASTA_F32, PASTA_BF16, PASTA_F16, PASTA_F64 = 0, 1, 2, 3
PASTA_CREATE_DEFAULT, PASTA_CREATE_NO_VALIDATE = 0, 1
MAX_ORDER = 8
MAX_RANK = 256
ALS_MAX_RANK = 128
OPS = {"add": 0, "sub": 1, "mul": 2, "div": 3}  # pasta_op

STATUS = {
    0: "PASTA_OK", 1: "PASTA_ERR_INVALID_ARG", 2: "PASTA_ERR_ALIGNMENT",
    3: "PASTA_ERR_INDEX_OOB", 4: "PASTA_ERR_NONFINITE", 5: "PASTA_ERR_NOT_SORTED",
    6: "PASTA_ERR_NOMEM", 7: "PASTA_ERR_CUDA", 8: "PASTA_ERR_UNSUPPORTED",
    9: "PASTA_ERR_SINGULAR",
}

# name -> (restype, argtypes); mirrors include/pasta.h
_P = ctypes.c_void_p
_I = ctypes.c_int
_U64 = ctypes.c_uint64
SIGNATURES = {
    "pasta_status_str": (ctypes.c_char_p, [_I]),
    "pasta_last_error": (ctypes.c_char_p, []),
    "pasta_version": (_I, []),
    "pasta_coo_create": (_I, [_P, _I, _P, _U64, _P, _P, ctypes.c_uint, _P]),
    "pasta_coo_destroy": (_I, [_P]),
    "pasta_coo_info": (_I, [_P, _P, _P, _P]),
    "pasta_coo_sort_by_mode": (_I, [_P, _I, _P]),
    "pasta_coo_view": (_I, [_P, _I, _P, _P, _P]),
    "pasta_coo_copy_out": (_I, [_P, _I, _P, _P, _P, _P]),
    "pasta_mttkrp": (_I, [_P, _P, _I, _I, _I, _P, _P]),
    "pasta_cp_loss_fwd": (_I, [_P, _P, _I, _I, _I, _P, _P, _P]),
    "pasta_cp_loss_bwd": (_I, [_P, _P, _I, _I, _I, _P, _P, _P]),
    "pasta_convert": (_I, [_P, _I, _P, _I, _U64, _P]),
    "pasta_convert_scaled": (_I, [_P, _I, _P, _I, _U64, _P, _P]),
    "pasta_cp_loss_fwd_bwd": (_I, [_P, _P, _I, _I, _P, _P, _P, _P]),
    "pasta_cp_loss_fwd_noalloc": (_I, [_I, _P, _U64, _P, _P, _P, _I, _I, _P, _P, _P]),
    "pasta_cp_als_sweep": (_I, [_P, _P, _I, _P, _P, _P]),
    "pasta_cp_als": (_I, [_P, _P, _I, _I, ctypes.c_double, _P, _P, _P, _P]),
    "pasta_tew_eq": (_I, [_P, _P, _I, _P, _P]),
    "pasta_ts": (_I, [_P, _I, ctypes.c_double, _P, _P]),
    "pasta_coo_fibers": (_I, [_P, _I, _P, _P]),
    "pasta_coo_fiber_coords": (_I, [_P, _I, _P, _P]),
    "pasta_ttm": (_I, [_P, _I, _P, _I, _I, _P, _P]),
    "pasta_ttv": (_I, [_P, _I, _P, _I, _P, _P]),
    "pasta_set_allocator": (_I, [_P, _P, _P]),
    "pasta_set_grid_cap": (_I, [_I]),
    "pasta_gather_probe": (_I, [_P, _P, _I, _I, _I, _P, _U64, _P]),
    "pasta_coo_hicoo": (_I, [_P, _I, _P, _P]),
    "pasta_mttkrp_range": (_I, [_P, _P, _I, _I, _I, _U64, _U64, _P, _P]),
    "pasta_cp_loss_fwd_bwd_range": (_I, [_P, _P, _I, _I, _U64, _U64, _P, _P, _P, _P]),
    "pasta_hicoo_copy_out": (_I, [_P, _P, _P, _P, _P, _P]),
    "pasta_hicoo_mttkrp": (_I, [_P, _P, _I, _I, _I, _P, _P]),
    "pasta_get_grid_cap": (_I, []),
    "pasta_memcpy": (_I, [_P, _P, _U64, _P]),
    "pasta_coo_create_sorted": (_I, [_P, _I, _P, _U64, _P, _P, ctypes.c_uint, _I, _P]),
}

_lock = threading.Lock()
_lib = None


class PastaError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        self.status = status
        self.name = STATUS.get(status, f"status {status}")
        super().__init__(f"{where}: {self.name}: {detail}")


def lib() -> ctypes.CDLL:
    """Load libpasta.so (built by ``paper_1902_03317_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    f"libpasta.so is not built ({LIB_PATH} missing); run "
                    "`python -c 'import __graft_entry__ as g; g.build()'` first")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def check(status: int, where: str) -> None:
    if status != 0:
        detail = lib().pasta_last_error().decode(errors="replace")
        raise PastaError(status, where, detail)


def ptr_array(ptrs) -> ctypes.Array:
    """A host array of device pointers (``const void* const*``)."""
    return (ctypes.c_void_p * len(ptrs))(*[p if p else None for p in ptrs])


def u64_array(vals) -> ctypes.Array:
    return (ctypes.c_uint64 * len(vals))(*[int(v) for v in vals])
