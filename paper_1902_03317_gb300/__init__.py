"""GB300-native COO MTTKRP, sparse CP loss, CP-ALS, TTV/TTM and TEW-eq/TS
(arXiv:1902.03317, PASTA).

The compute path is libpasta, a C-ABI CUDA library for sm_103a
(``include/pasta.h``); this package holds its build script, a ctypes binding
and a thin torch-facing API.  Nothing here computes on the CPU: if the
library is missing, calls fail with a RuntimeError.
"""
from .api import (CooTensor, CPLoss, acc_dtype, convert, copy_, cp_als, cp_als_sweep, cp_loss,  # noqa: F401
                  cp_loss_bwd, cp_loss_fwd, cp_loss_fwd_bwd, fiber_coords, fibers, gather_probe, grid_cap, hicoo,
                  hicoo_copy_out, hicoo_mttkrp, mttkrp, mttkrp_range, cp_loss_fwd_bwd_range,
                  tew_eq, ts, ttm, ttv, use_torch_allocator)
from ._lib import PastaError  # noqa: F401

__all__ = ["CooTensor", "CPLoss", "cp_loss", "cp_loss_fwd", "cp_loss_bwd", "cp_loss_fwd_bwd", "mttkrp",
           "cp_als_sweep", "cp_als", "tew_eq", "ts", "fibers", "fiber_coords", "ttm", "ttv", "convert",
           "acc_dtype", "use_torch_allocator", "grid_cap", "gather_probe", "hicoo", "hicoo_copy_out",
           "hicoo_mttkrp", "mttkrp_range", "cp_loss_fwd_bwd_range", "copy_", "PastaError"]
