"""pasta_cp_loss_fwd_noalloc through the C ABI (collected last on purpose).

This entry point serves callers that must not allocate device memory where
they compute the loss (inside another framework's stream capture, in
real-time or callback code, or next to a foreign allocator): it reads the
caller's own arrays and keeps its scratch in a fixed device array inside the
library.  Its results must match pasta_cp_loss_fwd on the same entries and
the FP64 oracle, on two calls in a row (the second call reuses the scratch
the first one left).  The cases cover the streaming kernel (FP32 R = 32,
BF16 R = 16 order 5) and the general kernel (FP32 R = 24, whose row is not a
power-of-two number of 16-byte slots, and FP64 factors).
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import paper_1902_03317_gb300 as pasta
from paper_1902_03317_gb300 import _lib, synth
from tests import _gpu as G

pytestmark = pytest.mark.gpu


def _padded(t: torch.Tensor) -> torch.Tensor:
    """A copy readable up to a multiple of 4 entries (the kernel's 16-byte loads)."""
    n = t.numel()
    buf = torch.zeros(((n + 3) // 4) * 4, dtype=t.dtype, device=t.device)
    buf[:n] = t
    return buf


@pytest.mark.parametrize("name,nnz,dims,R,dtype", [
    ("zipf3d", 200_001, (20_000, 10_000, 4_000), 32, torch.float32),
    ("zipf5d", 100_003, (8, 50_000, 10_000, 1_000, 100), 16, torch.bfloat16),
    ("zipf3d", 60_001, (5_000, 3_000, 1_000), 24, torch.float32),
    ("zipf3d", 20_003, (2_000, 1_000, 500), 5, torch.float32),     # R * 4 B not a multiple of 16: general kernel
    ("zipf4d", 30_002, (900, 800, 70, 20), 8, torch.float64),      # FP64: general kernel
])
def test_noalloc_loss_matches_handle_path(name, nnz, dims, R, dtype):
    Xh = synth.generate(G.small(name, nnz, dims))
    X = G.to_device(Xh)
    _, Us, rounded = G.factors(dims, R, 21, dtype)
    ref_loss, ref_e = pasta.cp_loss_fwd(X, Us, -1, want_resid=True)
    ref_loss = ref_loss.item()
    ref_e = ref_e.cpu().numpy()
    idx_h, val_h = G.host(Xh)
    o_loss, o_e = oracle.cp_loss(dims, idx_h, val_h, rounded, want_resid=True)
    tol = 1e-12 if dtype == torch.float64 else G.FP32_TOL
    rdt = torch.float64 if dtype == torch.float64 else torch.float32

    idx = [_padded(i.to(G.DEV)) for i in Xh.idx]
    val = _padded(Xh.val.to(G.DEV))
    lib = _lib.lib()
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        loss = torch.full((), float("nan"), dtype=torch.float64, device=G.DEV)
        e = torch.full((nnz,), float("nan"), dtype=rdt, device=G.DEV)
        st = lib.pasta_cp_loss_fwd_noalloc(
            len(dims), _lib.u64_array(dims), nnz, _lib.ptr_array([t.data_ptr() for t in idx]),
            val.data_ptr(), _lib.ptr_array([u.data_ptr() for u in Us]), pasta.api.pasta_dtype(dtype),
            R, loss.data_ptr(), e.data_ptr(), stream)
        _lib.check(st, "pasta_cp_loss_fwd_noalloc")
        torch.cuda.synchronize()
        assert abs(loss.item() - ref_loss) <= tol * ref_loss, call
        assert G.rel_err(e.cpu().numpy(), ref_e) < tol, call
        assert abs(loss.item() - o_loss) <= tol * o_loss, call
        assert G.rel_err(e.cpu().numpy(), o_e) < tol, call
    X.close()


def test_noalloc_rejects_bad_sizes_and_alignment():
    lib = _lib.lib()
    dims = [10, 10, 10]
    idx = [torch.zeros(8, dtype=torch.int32, device=G.DEV) for _ in dims]
    val = torch.zeros(8, device=G.DEV)
    U = [torch.zeros((10, 16), device=G.DEV) for _ in dims]
    loss = torch.zeros((), dtype=torch.float64, device=G.DEV)
    ptrs = _lib.ptr_array([t.data_ptr() for t in idx])
    uptr = _lib.ptr_array([u.data_ptr() for u in U])

    def call(order=3, d=dims, nnz=4, ip=ptrs, vp=val.data_ptr(), R=16):
        return _lib.STATUS[lib.pasta_cp_loss_fwd_noalloc(order, _lib.u64_array(d), nnz, ip, vp, uptr, 0,
                                                         R, loss.data_ptr(), None, None)]
    assert call() == "PASTA_OK"
    assert call(order=9, d=dims * 3) == "PASTA_ERR_INVALID_ARG"
    assert call(R=257) == "PASTA_ERR_INVALID_ARG"
    assert call(nnz=0xFFFF0000) == "PASTA_ERR_INVALID_ARG"
    assert call(vp=val.data_ptr() + 4) == "PASTA_ERR_ALIGNMENT"
    mis = _lib.ptr_array([idx[0].data_ptr(), idx[1].data_ptr() + 4, idx[2].data_ptr()])
    assert call(ip=mis) == "PASTA_ERR_ALIGNMENT"
    torch.cuda.synchronize()


def test_noalloc_call_allocates_nothing():
    """After the first call on the device (which looks up the scratch array's
    address), further calls change neither the device's free memory nor the
    allocation count of torch's caching allocator (which the library's own
    buffers would go through)."""
    nnz, dims, R = 50_000, (5_000, 3_000, 1_000), 32
    Xh = synth.generate(G.small("zipf3d", nnz, dims))
    _, Us, _ = G.factors(dims, R, 23)
    idx = [_padded(i.to(G.DEV)) for i in Xh.idx]
    val = _padded(Xh.val.to(G.DEV))
    loss = torch.zeros((), dtype=torch.float64, device=G.DEV)
    e = torch.zeros(nnz, dtype=torch.float32, device=G.DEV)
    lib = _lib.lib()

    def call():
        st = lib.pasta_cp_loss_fwd_noalloc(
            3, _lib.u64_array(dims), nnz, _lib.ptr_array([t.data_ptr() for t in idx]), val.data_ptr(),
            _lib.ptr_array([u.data_ptr() for u in Us]), 0, R, loss.data_ptr(), e.data_ptr(),
            torch.cuda.current_stream().cuda_stream)
        _lib.check(st, "pasta_cp_loss_fwd_noalloc")

    call()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    n0 = torch.cuda.memory_stats().get("allocation.all.allocated", 0)
    for _ in range(3):
        call()
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.cuda.memory_stats().get("allocation.all.allocated", 0) == n0
