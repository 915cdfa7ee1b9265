"""Python API over libpasta: COO handles, MTTKRP, the CP loss and its
autograd, CP-ALS, TEW-eq/TS and TTV/TTM.

PyTorch supplies device memory (its caching allocator also backs the
library's own buffers) and the current CUDA stream; every step of the
computation (copy-in and validation, mode sort, MTTKRP, loss forward and
backward, gradient down-conversion, the ALS solve, the element-wise and
mode-n products) runs in libpasta's kernels.  Operations follow
arXiv:1902.03317 (PASTA): COO storage (Sec. 5.1), mode-order sorting
(Sec. 5.2.2), MTTKRP (Eq. (mttkrp-init), Algorithm 6), the CP model behind
gradient-descent and ALS CPD (Sec. 2.2), TEW-eq/TS (Sec. 3.1, 3.2;
Algorithms 1, 3) and TTV/TTM (Sec. 3.3, 3.4; Algorithms 4, 5).
"""
from __future__ import annotations

import ctypes
from typing import Sequence

import torch

from . import _lib

_DTYPES = {
    torch.float32: _lib.PASTA_F32,
    torch.bfloat16: _lib.PASTA_BF16,
    torch.float16: _lib.PASTA_F16,
    torch.float64: _lib.PASTA_F64,
}


def pasta_dtype(dt: torch.dtype) -> int:
    try:
        return _DTYPES[dt]
    except KeyError:
        raise TypeError(f"unsupported factor dtype {dt}") from None


def acc_dtype(dt: torch.dtype) -> torch.dtype:
    """Output/accumulation dtype for factors of dtype ``dt``."""
    return torch.float64 if dt == torch.float64 else torch.float32


def _stream(device) -> int:
    return torch.cuda.current_stream(device).cuda_stream


# The library's own device buffers (stored copies, scratch, fiber tables) go
# through torch's caching allocator (pasta_set_allocator), so handles built
# and dropped in a loop reuse memory and torch's memory accounting sees them.
_ALLOC_T = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p)
_FREE_T = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


def _torch_alloc(nbytes, device, stream, ctx):
    try:
        return torch.cuda.caching_allocator_alloc(int(nbytes), int(device), int(stream or 0))
    except Exception:  # out of memory: the library reports PASTA_ERR_NOMEM
        return None


def _torch_free(ptr, ctx):
    torch.cuda.caching_allocator_delete(int(ptr))


_TORCH_CALLBACKS = (_ALLOC_T(_torch_alloc), _FREE_T(_torch_free))
_allocator = None  # None until the first handle; then "torch" or "cuda"


def use_torch_allocator(enable: bool = True) -> None:
    """Route the library's device buffers through torch's caching allocator
    (the default from the first handle on) or back to cudaMalloc.  Only
    possible while no library buffer is held."""
    global _allocator
    L = _lib.lib()
    if enable:
        st = L.pasta_set_allocator(ctypes.cast(_TORCH_CALLBACKS[0], ctypes.c_void_p),
                                   ctypes.cast(_TORCH_CALLBACKS[1], ctypes.c_void_p), None)
    else:
        st = L.pasta_set_allocator(None, None, None)
    _lib.check(st, "pasta_set_allocator")
    _allocator = "torch" if enable else "cuda"


def _ensure_allocator() -> None:
    if _allocator is None:
        use_torch_allocator(True)


class CooTensor:
    """A COO tensor held by libpasta on one CUDA device (``pasta_coo``).

    ``idx``: one int32/uint32-valued tensor of nnz indices per mode (0-based,
    Sec. 5.1); ``val``: nnz FP32 values.  The data is copied into
    library-owned, padded SoA arrays; the inputs may be freed afterwards.
    The inputs may be CUDA tensors or host tensors (then ``device`` names the
    CUDA device, default the current one): pinned host tensors are copied
    asynchronously on the current stream straight into the library's copy.
    ``sort_mode``: also build that mode's sorted copy in the same call
    (``pasta_coo_create_sorted``, which overlaps the copy-in with the sort).
    """

    def __init__(self, dims: Sequence[int], idx: Sequence[torch.Tensor], val: torch.Tensor,
                 validate: bool = True, device=None, sort_mode: int | None = None):
        dims = [int(d) for d in dims]
        order = len(dims)
        if len(idx) != order:
            raise ValueError("need one index tensor per mode")
        if val.is_cuda:
            self.device = val.device
        else:
            # host tensors (pinned: copied asynchronously straight into the
            # handle's copy; they are kept referenced until close())
            self.device = torch.device(device) if device is not None else torch.device(
                "cuda", torch.cuda.current_device())
            if self.device.type != "cuda":
                raise ValueError("device must be a CUDA device")
        self.dims = tuple(dims)
        self.order = order
        self.nnz = int(val.numel())
        idx_c = []
        for ix in idx:
            if ix.device != val.device or ix.numel() != self.nnz:
                raise ValueError("index tensors must be on val's device with nnz elements")
            if ix.dtype not in (torch.int32, torch.uint32):
                raise TypeError("indices must be int32 (values < 2^31) or uint32")
            idx_c.append(ix.contiguous())
        val_c = val.contiguous()
        if val_c.dtype != torch.float32:
            raise TypeError("values must be float32")
        _ensure_allocator()
        h = ctypes.c_void_p()
        flags = _lib.PASTA_CREATE_DEFAULT if validate else _lib.PASTA_CREATE_NO_VALIDATE
        with torch.cuda.device(self.device):
            if sort_mode is None:
                st = _lib.lib().pasta_coo_create(
                    ctypes.byref(h), order, _lib.u64_array(dims), self.nnz,
                    _lib.ptr_array([t.data_ptr() for t in idx_c]), val_c.data_ptr(), flags,
                    _stream(self.device))
            else:
                # create and sort `sort_mode` in one call (pasta_coo_create_sorted:
                # copy-in and sort overlapped for large pinned host inputs)
                st = _lib.lib().pasta_coo_create_sorted(
                    ctypes.byref(h), order, _lib.u64_array(dims), self.nnz,
                    _lib.ptr_array([t.data_ptr() for t in idx_c]), val_c.data_ptr(), flags,
                    int(sort_mode), _stream(self.device))
        _lib.check(st, "pasta_coo_create" if sort_mode is None else "pasta_coo_create_sorted")
        self._h = h
        self._sorted: set[int] = set() if sort_mode is None else {int(sort_mode)}
        self._host_refs = None if val.is_cuda else (idx_c, val_c)

    @property
    def handle(self) -> ctypes.c_void_p:
        if self._h is None:
            raise RuntimeError("CooTensor is closed")
        return self._h

    @classmethod
    def _adopt(cls, handle: ctypes.c_void_p, like: "CooTensor") -> "CooTensor":
        """Wrap a handle the library created with ``like``'s order, dims and nnz."""
        t = cls.__new__(cls)
        t.device, t.dims, t.order, t.nnz = like.device, like.dims, like.order, like.nnz
        t._h = handle
        t._sorted = set()
        t._host_refs = None
        return t

    def close(self) -> None:
        if getattr(self, "_h", None) is not None:
            _lib.lib().pasta_coo_destroy(self._h)  # synchronises the device
            self._h = None
        self._host_refs = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sort_by_mode(self, mode: int) -> "CooTensor":
        """Build the mode-``mode`` sorted copy (Sec. 5.2.2) if not present."""
        if mode not in self._sorted:
            with torch.cuda.device(self.device):
                st = _lib.lib().pasta_coo_sort_by_mode(self.handle, int(mode), _stream(self.device))
            _lib.check(st, "pasta_coo_sort_by_mode")
            self._sorted.add(int(mode))
        return self

    def sort_all(self) -> "CooTensor":
        """Build every mode's sorted copy, in the order 0, N-1, ..., 1: each
        copy after the first is then sorted from the next mode's copy on its
        own index field only."""
        for n in [0] + list(range(self.order - 1, 0, -1)):
            self.sort_by_mode(n)
        return self

    def copy_out(self, mode: int = -1):
        """Device copies of one stored copy: (idx list int32, val, perm or None)."""
        idx = [torch.empty(self.nnz, dtype=torch.int32, device=self.device) for _ in range(self.order)]
        val = torch.empty(self.nnz, dtype=torch.float32, device=self.device)
        perm = None if mode < 0 else torch.empty(self.nnz, dtype=torch.int32, device=self.device)
        with torch.cuda.device(self.device):
            st = _lib.lib().pasta_coo_copy_out(
                self.handle, int(mode), _lib.ptr_array([t.data_ptr() for t in idx]),
                val.data_ptr(), perm.data_ptr() if perm is not None else None,
                _stream(self.device))
        _lib.check(st, "pasta_coo_copy_out")
        return idx, val, perm


def _elementwise_out(X: CooTensor, out: CooTensor | None):
    if out is None:
        return ctypes.c_void_p(), None
    if out is X:
        raise ValueError("out must differ from the inputs")
    out._sorted.clear()  # the library drops the output's sorted copies
    return ctypes.c_void_p(out.handle.value), out


def tew_eq(X: CooTensor, Y: CooTensor, op: str, out: CooTensor | None = None) -> CooTensor:
    """Z = X op Y (``op`` in add/sub/mul/div) for tensors storing the same
    coordinates in the same order (TEW-eq, Algorithm 1).  Returns a new
    CooTensor, or writes ``out`` (same shape, neither input) and returns it."""
    h, o = _elementwise_out(X, out)
    if o is Y:
        raise ValueError("out must differ from the inputs")
    with torch.cuda.device(X.device):
        st = _lib.lib().pasta_tew_eq(X.handle, Y.handle, _lib.OPS[op], ctypes.byref(h), _stream(X.device))
    _lib.check(st, "pasta_tew_eq")
    return o if o is not None else CooTensor._adopt(h, X)


def ts(X: CooTensor, op: str, s: float, out: CooTensor | None = None) -> CooTensor:
    """Z = X op s for every stored value (TS, Algorithm 3), FP32 with s
    rounded to FP32.  Returns a new CooTensor or writes ``out``."""
    h, o = _elementwise_out(X, out)
    with torch.cuda.device(X.device):
        st = _lib.lib().pasta_ts(X.handle, _lib.OPS[op], float(s), ctypes.byref(h), _stream(X.device))
    _lib.check(st, "pasta_ts")
    return o if o is not None else CooTensor._adopt(h, X)


def fibers(X: CooTensor, mode: int) -> int:
    """Build (once) the mode-``mode`` fiber table (sorting mode (mode+1) % N
    first if needed); returns the number of fibers."""
    X.sort_by_mode((mode + 1) % X.order)
    n = ctypes.c_uint64()
    with torch.cuda.device(X.device):
        st = _lib.lib().pasta_coo_fibers(X.handle, int(mode), ctypes.byref(n), _stream(X.device))
    _lib.check(st, "pasta_coo_fibers")
    return int(n.value)


def fiber_coords(X: CooTensor, mode: int) -> list[torch.Tensor]:
    """The mode-``mode`` fibers' coordinates in modes mode+1, ..., mode-1
    (cyclic): N-1 int32 tensors of nfibs."""
    nf = fibers(X, mode)
    out = [torch.empty(nf, dtype=torch.int32, device=X.device) for _ in range(X.order - 1)]
    with torch.cuda.device(X.device):
        st = _lib.lib().pasta_coo_fiber_coords(X.handle, int(mode), _lib.ptr_array([t.data_ptr() for t in out]),
                                               _stream(X.device))
    _lib.check(st, "pasta_coo_fiber_coords")
    return out


def ttm(X: CooTensor, U: torch.Tensor, mode: int) -> torch.Tensor:
    """Y = X x_mode U (Algorithm 5; U is dims[mode] x R): one row per mode-n
    fiber, in the order of ``fiber_coords``.  FP32 result (FP64 for FP64 U)."""
    nf = fibers(X, mode)
    if U.dim() != 2 or U.shape[0] != X.dims[mode] or not U.is_contiguous() or U.device != X.device:
        raise ValueError(f"U must be a contiguous {X.dims[mode]} x R tensor on the tensor's device")
    R = int(U.shape[1])
    Y = torch.empty((nf, R), dtype=acc_dtype(U.dtype), device=X.device)
    with torch.cuda.device(X.device):
        st = _lib.lib().pasta_ttm(X.handle, int(mode), U.data_ptr(), pasta_dtype(U.dtype), R, Y.data_ptr(),
                                  _stream(X.device))
    _lib.check(st, "pasta_ttm")
    return Y


def ttv(X: CooTensor, v: torch.Tensor, mode: int) -> torch.Tensor:
    """y = X x_mode v (Algorithm 4): one value per mode-n fiber."""
    nf = fibers(X, mode)
    if v.dim() != 1 or v.shape[0] != X.dims[mode] or not v.is_contiguous() or v.device != X.device:
        raise ValueError(f"v must be a contiguous vector of {X.dims[mode]} on the tensor's device")
    y = torch.empty(nf, dtype=acc_dtype(v.dtype), device=X.device)
    with torch.cuda.device(X.device):
        st = _lib.lib().pasta_ttv(X.handle, int(mode), v.data_ptr(), pasta_dtype(v.dtype), y.data_ptr(),
                                  _stream(X.device))
    _lib.check(st, "pasta_ttv")
    return y


def _factor_ptrs(X: CooTensor, Us: Sequence[torch.Tensor | None], skip: int = -1):
    if len(Us) != X.order:
        raise ValueError("need one factor per mode")
    dt = None
    R = None
    ptrs = []
    for k, U in enumerate(Us):
        if U is None:
            if k != skip:
                raise ValueError(f"factor {k} is required")
            ptrs.append(None)
            continue
        if U.device != X.device or U.dim() != 2 or U.shape[0] != X.dims[k]:
            raise ValueError(f"factor {k} must be a {X.dims[k]} x R tensor on {X.device}")
        if not U.is_contiguous():
            raise ValueError(f"factor {k} must be contiguous (row-major)")
        if dt is None:
            dt, R = U.dtype, int(U.shape[1])
        elif U.dtype != dt or int(U.shape[1]) != R:
            raise ValueError("all factors must share dtype and R")
        ptrs.append(U.data_ptr())
    return _lib.ptr_array(ptrs), dt, R


def mttkrp(X: CooTensor, Us: Sequence[torch.Tensor | None], mode: int,
           out: torch.Tensor | None = None) -> torch.Tensor:
    """Mode-``mode`` MTTKRP (Eq. (mttkrp-init)); ``Us[mode]`` may be None.
    Sorts for ``mode`` first if needed.  Returns ``dims[mode] x R`` in FP32
    (FP64 for FP64 factors)."""
    X.sort_by_mode(mode)
    ptrs, dt, R = _factor_ptrs(X, Us, skip=mode)
    if out is None:
        out = torch.empty((X.dims[mode], R), dtype=acc_dtype(dt), device=X.device)
    elif out.shape != (X.dims[mode], R) or out.dtype != acc_dtype(dt) or not out.is_contiguous():
        raise ValueError("bad out tensor")
    with torch.cuda.device(X.device):
        st = _lib.lib().pasta_mttkrp(X.handle, ptrs, pasta_dtype(dt), int(mode), R,
                                     out.data_ptr(), _stream(X.device))
    _lib.check(st, "pasta_mttkrp")
    return out


def mttkrp_range(X: CooTensor, Us: Sequence[torch.Tensor | None], mode: int, lo: int, hi: int,
                 out: torch.Tensor | None = None) -> torch.Tensor:
    """MTTKRP over the entries at positions [lo, hi) of the mode-``mode``
    sorted copy (pasta_mttkrp_range; lo a multiple of 4).  Outputs of ranges
    that partition the copy sum to ``mttkrp``'s."""
    X.sort_by_mode(mode)
    ptrs, dt, R = _factor_ptrs(X, Us, skip=mode)
    if out is None:
        out = torch.empty((X.dims[mode], R), dtype=acc_dtype(dt), device=X.device)
    with torch.cuda.device(X.device):
        st = _lib.lib().pasta_mttkrp_range(X.handle, ptrs, pasta_dtype(dt), int(mode), R, int(lo), int(hi),
                                           out.data_ptr(), _stream(X.device))
    _lib.check(st, "pasta_mttkrp_range")
    return out


def cp_loss_fwd_bwd_range(X: CooTensor, Us: Sequence[torch.Tensor], lo: int, hi: int,
                          gscale: torch.Tensor | None = None):
    """Loss and gradients over positions [lo, hi) of every sorted copy
    (pasta_cp_loss_fwd_bwd_range); sums over ranges that partition the
    entries give ``cp_loss_fwd_bwd``'s results."""
    X.sort_all()
    ptrs, dt, R = _factor_ptrs(X, Us)
    loss = torch.empty((), dtype=torch.float64, device=X.device)
    G = [torch.empty((d, R), dtype=acc_dtype(dt), device=X.device) for d in X.dims]
    gp = None
    if gscale is not None:
        gscale = gscale.to(device=X.device, dtype=torch.float64).reshape(()).contiguous()
        gp = gscale.data_ptr()
    with torch.cuda.device(X.device):
        st = _lib.lib().pasta_cp_loss_fwd_bwd_range(X.handle, ptrs, pasta_dtype(dt), R, int(lo), int(hi),
                                                    loss.data_ptr(), gp,
                                                    _lib.ptr_array([g.data_ptr() for g in G]), _stream(X.device))
    _lib.check(st, "pasta_cp_loss_fwd_bwd_range")
    return loss, G


def hicoo(X: CooTensor, block_bits: int = 7) -> int:
    """Build the HiCOO copy of ``X`` (pasta_coo_hicoo: blocks of
    2^block_bits cells per mode, one offset byte per mode per entry; one copy
    for every mode).  Returns the number of nonempty blocks."""
    nb = ctypes.c_uint64()
    with torch.cuda.device(X.device):
        st = _lib.lib().pasta_coo_hicoo(X.handle, int(block_bits), ctypes.byref(nb), _stream(X.device))
    _lib.check(st, "pasta_coo_hicoo")
    return int(nb.value)


def hicoo_copy_out(X: CooTensor, nblocks: int):
    """The HiCOO arrays as device tensors: (bptr[nb + 1] int32, binds: list of
    N int32 [nb], einds: list of N uint8 [nnz], val float32 [nnz])."""
    dev = X.device
    bptr = torch.empty(nblocks + 1, dtype=torch.int32, device=dev)
    binds = [torch.empty(nblocks, dtype=torch.int32, device=dev) for _ in X.dims]
    einds = [torch.empty(X.nnz, dtype=torch.uint8, device=dev) for _ in X.dims]
    val = torch.empty(X.nnz, dtype=torch.float32, device=dev)
    with torch.cuda.device(dev):
        st = _lib.lib().pasta_hicoo_copy_out(X.handle, bptr.data_ptr(),
                                             _lib.ptr_array([b.data_ptr() for b in binds]),
                                             _lib.ptr_array([e.data_ptr() for e in einds]),
                                             val.data_ptr(), _stream(dev))
    _lib.check(st, "pasta_hicoo_copy_out")
    return bptr, binds, einds, val


def hicoo_mttkrp(X: CooTensor, Us: Sequence[torch.Tensor | None], mode: int,
                 out: torch.Tensor | None = None) -> torch.Tensor:
    """Mode-``mode`` MTTKRP from the HiCOO copy (built first with ``hicoo``).
    Same result as ``mttkrp`` up to FP32 rounding."""
    ptrs, dt, R = _factor_ptrs(X, Us, skip=mode)
    if out is None:
        out = torch.empty((X.dims[mode], R), dtype=acc_dtype(dt), device=X.device)
    with torch.cuda.device(X.device):
        st = _lib.lib().pasta_hicoo_mttkrp(X.handle, ptrs, pasta_dtype(dt), int(mode), R, out.data_ptr(),
                                           _stream(X.device))
    _lib.check(st, "pasta_hicoo_mttkrp")
    return out


def gather_probe(X: CooTensor, Us: Sequence[torch.Tensor | None], mode: int,
                 sink: torch.Tensor | None = None) -> torch.Tensor:
    """Diagnostic: the row gathers of ``mttkrp(X, Us, mode)`` alone (same
    kernel and launch, no arithmetic into output rows); returns the FP32
    sink it wrote (one float per thread, meaningless values).  Its time is
    the gather ceiling of the MTTKRP on this tensor."""
    X.sort_by_mode(mode)
    ptrs, dt, R = _factor_ptrs(X, Us, skip=mode)
    if sink is None:
        sink = torch.empty(1 << 22, dtype=torch.float32, device=X.device)
    with torch.cuda.device(X.device):
        st = _lib.lib().pasta_gather_probe(X.handle, ptrs, pasta_dtype(dt), int(mode), R,
                                           sink.data_ptr(), sink.numel(), _stream(X.device))
    _lib.check(st, "pasta_gather_probe")
    return sink


def cp_loss_fwd(X: CooTensor, Us: Sequence[torch.Tensor], mode: int = -1,
                want_resid: bool = False):
    """Sparse CP least-squares loss over the stored entries (FP64 0-d tensor),
    optionally with the residuals in the order of the streamed copy."""
    if mode >= 0:
        X.sort_by_mode(mode)
    ptrs, dt, R = _factor_ptrs(X, Us)
    loss = torch.empty((), dtype=torch.float64, device=X.device)
    resid = torch.empty(X.nnz, dtype=acc_dtype(dt), device=X.device) if want_resid else None
    with torch.cuda.device(X.device):
        st = _lib.lib().pasta_cp_loss_fwd(X.handle, ptrs, pasta_dtype(dt), R, int(mode),
                                          loss.data_ptr(),
                                          resid.data_ptr() if resid is not None else None,
                                          _stream(X.device))
    _lib.check(st, "pasta_cp_loss_fwd")
    return (loss, resid) if want_resid else loss


BWD_PER_MODE = -2


def cp_loss_bwd(X: CooTensor, Us: Sequence[torch.Tensor], mode: int = BWD_PER_MODE,
                gscale: torch.Tensor | None = None) -> list[torch.Tensor]:
    """Gradient of ``gscale * loss`` for every factor; FP32 (FP64 for FP64
    factors) accumulators.  ``mode``: -1 one pass over the creation-order copy
    (atomics), n one pass over the mode-n copy (mode n reduced along runs,
    atomics for the others), -2 (default) one pass per mode over its own
    sorted copy (run reduction only; no contention on hot rows)."""
    if mode == BWD_PER_MODE:
        X.sort_all()
    elif mode >= 0:
        X.sort_by_mode(mode)
    ptrs, dt, R = _factor_ptrs(X, Us)
    G = [torch.empty((d, R), dtype=acc_dtype(dt), device=X.device) for d in X.dims]
    gp = None
    if gscale is not None:
        gscale = gscale.to(device=X.device, dtype=torch.float64).contiguous()
        gp = gscale.data_ptr()
    with torch.cuda.device(X.device):
        st = _lib.lib().pasta_cp_loss_bwd(X.handle, ptrs, pasta_dtype(dt), R, int(mode), gp,
                                          _lib.ptr_array([g.data_ptr() for g in G]),
                                          _stream(X.device))
    _lib.check(st, "pasta_cp_loss_bwd")
    return G


def convert(src: torch.Tensor, dtype: torch.dtype, scale: torch.Tensor | None = None,
            out: torch.Tensor | None = None) -> torch.Tensor:
    """Element-wise ``(dtype)(scale * src)`` in libpasta (round to nearest
    even); ``scale`` is an optional device scalar.  ``out`` may be ``src``
    itself when the dtypes agree (in place)."""
    src = src.contiguous()
    if out is None:
        out = torch.empty(src.shape, dtype=dtype, device=src.device)
    sp = None
    if scale is not None:
        scale = scale.to(device=src.device, dtype=torch.float64).reshape(()).contiguous()
        sp = scale.data_ptr()
    with torch.cuda.device(src.device):
        st = _lib.lib().pasta_convert_scaled(src.data_ptr(), pasta_dtype(src.dtype), out.data_ptr(),
                                             pasta_dtype(dtype), src.numel(), sp,
                                             _stream(src.device))
    _lib.check(st, "pasta_convert_scaled")
    return out


def cp_loss_fwd_bwd(X: CooTensor, Us: Sequence[torch.Tensor],
                    gscale: torch.Tensor | None = None):
    """Loss and the gradients of ``gscale * loss`` in N passes (one per mode,
    the first also summing the loss).  Returns (FP64 loss, list of FP32
    gradients; FP64 for FP64 factors)."""
    X.sort_all()
    ptrs, dt, R = _factor_ptrs(X, Us)
    loss = torch.empty((), dtype=torch.float64, device=X.device)
    G = [torch.empty((d, R), dtype=acc_dtype(dt), device=X.device) for d in X.dims]
    gp = None
    if gscale is not None:
        gscale = gscale.to(device=X.device, dtype=torch.float64).reshape(()).contiguous()
        gp = gscale.data_ptr()
    with torch.cuda.device(X.device):
        st = _lib.lib().pasta_cp_loss_fwd_bwd(X.handle, ptrs, pasta_dtype(dt), R, loss.data_ptr(),
                                              gp, _lib.ptr_array([g.data_ptr() for g in G]),
                                              _stream(X.device))
    _lib.check(st, "pasta_cp_loss_fwd_bwd")
    return loss, G


def cp_als_sweep(X: CooTensor, Us: Sequence[torch.Tensor], want_fit: bool = True):
    """One CP-ALS sweep (pasta_cp_als_sweep): updates the FP32 factors ``Us``
    in place, mode 0 first; returns ``(lam, fit)`` as FP64 device tensors
    (``fit`` None when ``want_fit`` is False).  Sorts every mode first.
    Raises PastaError (PASTA_ERR_SINGULAR) when a normal-equation matrix has
    no inverse."""
    X.sort_all()
    R = int(Us[0].shape[1])
    for k, U in enumerate(Us):
        if U.dtype != torch.float32 or not U.is_contiguous() or U.device != X.device:
            raise ValueError("CP-ALS factors must be contiguous FP32 tensors on the tensor's device")
        if tuple(U.shape) != (X.dims[k], R):
            raise ValueError(f"U[{k}] must be {X.dims[k]} x {R}")
    lam = torch.empty(R, dtype=torch.float64, device=X.device)
    fit = torch.empty((), dtype=torch.float64, device=X.device) if want_fit else None
    with torch.cuda.device(X.device):
        st = _lib.lib().pasta_cp_als_sweep(X.handle, _lib.ptr_array([U.data_ptr() for U in Us]), R,
                                           lam.data_ptr(), fit.data_ptr() if want_fit else None,
                                           _stream(X.device))
    _lib.check(st, "pasta_cp_als_sweep")
    return lam, fit


def cp_als(X: CooTensor, R: int, max_sweeps: int = 50, tol: float = 1e-5,
           init: Sequence[torch.Tensor] | None = None, seed: int = 0):
    """CP decomposition by alternating least squares (pasta_cp_als): sweeps
    until the fit changes by less than ``tol`` or ``max_sweeps`` is reached
    (``tol < 0``: always ``max_sweeps``).  ``init`` defaults to N(0, 1)
    factors drawn on the device from ``seed``.  Returns ``(Us, lam, fits)``
    with the fit after each sweep run."""
    if init is None:
        g = torch.Generator(device=X.device).manual_seed(seed)
        Us = [torch.randn((d, R), generator=g, device=X.device, dtype=torch.float32) for d in X.dims]
    else:
        Us = [u.detach().to(device=X.device, dtype=torch.float32).contiguous().clone() for u in init]
    X.sort_all()
    for k, U in enumerate(Us):
        if tuple(U.shape) != (X.dims[k], R):
            raise ValueError(f"U[{k}] must be {X.dims[k]} x {R}")
    lam = torch.empty(R, dtype=torch.float64, device=X.device)
    fits = (ctypes.c_double * max(1, int(max_sweeps)))()
    done = ctypes.c_int(0)
    with torch.cuda.device(X.device):
        st = _lib.lib().pasta_cp_als(X.handle, _lib.ptr_array([U.data_ptr() for U in Us]), int(R), int(max_sweeps),
                                     float(tol), lam.data_ptr(), ctypes.cast(fits, ctypes.c_void_p),
                                     ctypes.cast(ctypes.pointer(done), ctypes.c_void_p), _stream(X.device))
    _lib.check(st, "pasta_cp_als")
    return Us, lam, [float(fits[i]) for i in range(done.value)]


class CPLoss(torch.autograd.Function):
    """loss = 1/2 sum_m (x_m - sum_r prod_k U_k(i_k(m), r))^2 over the stored
    entries of X, with hand-written forward and backward kernels.

    ``CPLoss.apply(X, mode, *Us)``: ``mode`` selects how the stored entries
    are streamed: -1 creation order; n the mode-n sorted copy (the backward
    reduces mode n along runs, the others with atomics); -2 (default of
    ``cp_loss``) the forward over the mode-0 copy and the backward as one pass
    per mode over each mode's sorted copy.  With -2 and any factor requiring a
    gradient, the forward already computes the gradients for g = 1 in the
    same N passes (pasta_cp_loss_fwd_bwd) and the backward only scales them
    by the incoming gradient.  Returns an FP64 0-d tensor; gradients come back
    in each factor's dtype (FP32 accumulation, converted on the device)."""

    @staticmethod
    def forward(ctx, X: CooTensor, mode: int, *Us: torch.Tensor):
        Us = [U.detach() for U in Us]
        ctx.X = X
        ctx.mode = mode
        ctx.dtypes = [U.dtype for U in Us]
        ctx.G = None
        ctx.save_for_backward(*Us)  # a second backward (retain_graph) recomputes
        if mode == BWD_PER_MODE and any(ctx.needs_input_grad[2:]):
            loss, ctx.G = cp_loss_fwd_bwd(X, Us)
            return loss
        return cp_loss_fwd(X, Us, 0 if mode == BWD_PER_MODE else mode)

    @staticmethod
    def backward(ctx, grad_out: torch.Tensor):
        g = grad_out.detach().reshape(())
        grads = []
        if ctx.G is not None:
            for dt, G in zip(ctx.dtypes, ctx.G):
                grads.append(convert(G, dt, scale=g, out=G if G.dtype == dt else None))
            ctx.G = None
        else:
            Us = ctx.saved_tensors
            mode = ctx.mode
            for U, G in zip(Us, cp_loss_bwd(ctx.X, Us, mode, gscale=g)):
                grads.append(G if G.dtype == U.dtype else convert(G, U.dtype))
        return (None, None, *grads)


def cp_loss(X: CooTensor, Us: Sequence[torch.Tensor], mode: int = BWD_PER_MODE) -> torch.Tensor:
    """Differentiable sparse CP loss (see CPLoss)."""
    return CPLoss.apply(X, mode, *Us)


class grid_cap:
    """Context manager limiting every MTTKRP / CP-loss launch to at most
    ``max_blocks`` thread blocks (``pasta_set_grid_cap``; 0 = no limit), so
    that small inputs walk the kernels' multi-round (grid-strided) path.
    Restores the previous cap on exit.  A diagnostic: results depend on it
    only through FP32 rounding."""

    def __init__(self, max_blocks: int):
        self.max_blocks = int(max_blocks)
        self._prev = 0

    def __enter__(self):
        L = _lib.lib()
        self._prev = L.pasta_get_grid_cap()
        _lib.check(L.pasta_set_grid_cap(self.max_blocks), "pasta_set_grid_cap")
        return self

    def __exit__(self, *exc):
        _lib.check(_lib.lib().pasta_set_grid_cap(self._prev), "pasta_set_grid_cap")
        return False


def copy_(dst: torch.Tensor, src: torch.Tensor) -> torch.Tensor:
    """``dst`` <- ``src`` through ``pasta_memcpy`` on the current stream of
    the CUDA tensor's device: same number of bytes, both contiguous; either
    may be a CUDA tensor or a host tensor.  Between pinned host memory and the
    GPU the SMs move the data instead of the copy engine.  Asynchronous like
    ``Tensor.copy_(..., non_blocking=True)``: keep host tensors alive and
    untouched until the stream has passed the copy.  Returns ``dst``."""
    if not (dst.is_contiguous() and src.is_contiguous()):
        raise ValueError("copy_ needs contiguous tensors")
    nbytes = dst.numel() * dst.element_size()
    if nbytes != src.numel() * src.element_size():
        raise ValueError("copy_ needs tensors of the same size in bytes")
    dev = dst.device if dst.is_cuda else src.device
    if dev.type != "cuda":
        raise ValueError("copy_ needs one CUDA tensor")
    with torch.cuda.device(dev):
        st = _lib.lib().pasta_memcpy(dst.data_ptr(), src.data_ptr(), nbytes, _stream(dev))
    _lib.check(st, "pasta_memcpy")
    return dst
