"""Fiber tables, TTV and TTM (pasta_coo_fibers, pasta_ttv, pasta_ttm) on the
GPU vs the FP64 oracle, and the order-2 MTTKRP they run on.

Fiber coordinates are integer work: bit-exact, in the same order.  Values:
each fiber's sum runs in FP32 like MTTKRP's row sums, so FP32 factors are
held to the MTTKRP bar (relative Frobenius 1e-5) and 16-bit factors to it
against the oracle run on the same rounded factors.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1902_03317_gb300 as pasta
from paper_1902_03317_gb300 import _lib, synth
from tests import _gpu as G

pytestmark = pytest.mark.gpu

CASES = [
    ("zipf3d", 300_001, (5_000, 3_000, 2_000)),
    ("zipf4d", 200_003, (2_000, 2_000, 500, 100)),      # duplicates kept
    ("zipf5d", 150_001, (8, 3_000, 2_000, 500, 100)),
    ("uniform3d_200", 20_000, (200, 200, 200)),
]


def _tensor(name, nnz, dims, seed=None):
    wl = G.small(name, nnz, dims, seed=seed)
    Xh = synth.generate(wl)
    idx, val = G.host(Xh)
    return wl, G.to_device(Xh), idx, val


@pytest.mark.parametrize("name,nnz,dims", CASES)
def test_fibers_and_ttm_match_oracle(name, nnz, dims):
    wl, X, idx, val = _tensor(name, nnz, dims)
    g = torch.Generator().manual_seed(9)
    for n in range(wl.order):
        for R, dtype in ((32, torch.float32), (5, torch.float32), (32, torch.bfloat16), (8, torch.float64)):
            master = torch.randn(wl.dims[n], R, generator=g, dtype=torch.float64)
            U = master.to(dtype).to(G.DEV).contiguous()
            Y = pasta.ttm(X, U, n)
            coords, ref = oracle.ttm(wl.dims, idx, val, U.double().cpu().numpy(), n)
            got_coords = pasta.fiber_coords(X, n)
            assert len(got_coords) == len(coords)
            for a, b in zip(got_coords, coords):
                assert np.array_equal(a.cpu().numpy().astype(np.uint32), b), (name, n)
            assert Y.shape == ref.shape
            tol = 1e-12 if dtype == torch.float64 else G.FP32_TOL
            err = G.rel_err(Y.cpu().numpy(), ref)
            assert err < tol, (name, n, R, dtype, err)
    X.close()


@pytest.mark.parametrize("name,nnz,dims", CASES)
def test_ttv_matches_oracle(name, nnz, dims):
    wl, X, idx, val = _tensor(name, nnz, dims)
    for n in range(wl.order):
        for dtype in (torch.float32, torch.bfloat16, torch.float64):
            v = torch.randn(wl.dims[n], dtype=torch.float64, device=G.DEV).to(dtype)
            y = pasta.ttv(X, v, n)
            coords, ref = oracle.ttv(wl.dims, idx, val, v.double().cpu().numpy(), n)
            tol = 1e-12 if dtype == torch.float64 else G.FP32_TOL
            assert G.rel_err(y.cpu().numpy(), ref) < tol, (name, n, dtype)
            assert pasta.fibers(X, n) == ref.shape[0]
    X.close()


@pytest.mark.parametrize("name,nnz,dims", CASES[:3])
def test_ttm_writes_every_output_element(name, nnz, dims):
    """TTM clears only the rows it adds into atomically (rows open at a
    group-tile end) and stores every other fiber's row whole, so an output
    buffer full of NaN must come back fully overwritten, equal to the oracle.
    zipf4d keeps duplicate coordinates: fibers long enough to span tiles."""
    wl, X, idx, val = _tensor(name, nnz, dims)
    L = _lib.lib()
    for n in range(wl.order):
        for R in (32, 8):
            U = torch.randn(wl.dims[n], R, device=G.DEV)
            nf = pasta.fibers(X, n)
            Y = torch.full((nf, R), float("nan"), device=G.DEV)
            st = L.pasta_ttm(X.handle, n, U.data_ptr(), pasta.api.pasta_dtype(U.dtype), R, Y.data_ptr(),
                             torch.cuda.current_stream().cuda_stream)
            _lib.check(st, "pasta_ttm")
            got = Y.cpu().numpy()
            assert not np.isnan(got).any(), (name, n, R)
            _, ref = oracle.ttm(wl.dims, idx, val, U.double().cpu().numpy(), n)
            assert G.rel_err(got, ref) < G.FP32_TOL, (name, n, R)
    X.close()


def test_order2_mttkrp_is_spmm():
    """Order-2 MTTKRP (the streaming kernel's N = 2 path): M = X V for a
    sparse matrix X, both modes, FP32 and BF16."""
    wl, X, idx, val = _tensor("zipf3d", 200_000, (3_000, 2_000, 1))
    X2 = pasta.CooTensor((3_000, 2_000), [torch.tensor(ix.astype(np.int32), device=G.DEV) for ix in idx[:2]],
                         torch.tensor(val, dtype=torch.float32, device=G.DEV))
    X2.sort_all()
    for dtype in (torch.float32, torch.bfloat16):
        Us = [torch.randn(d, 32, device=G.DEV).to(dtype) for d in (3_000, 2_000)]
        for n in range(2):
            M = pasta.mttkrp(X2, Us, n)
            ref = oracle.mttkrp((3_000, 2_000), idx[:2], val, [u.double().cpu().numpy() for u in Us], n)
            assert G.rel_err(M.cpu().numpy(), ref) < G.FP32_TOL
    X.close()
    X2.close()


def test_edge_cases():
    # one stored entry
    X = pasta.CooTensor((4, 5, 6), [torch.tensor([1], dtype=torch.int32, device=G.DEV),
                                    torch.tensor([2], dtype=torch.int32, device=G.DEV),
                                    torch.tensor([3], dtype=torch.int32, device=G.DEV)],
                        torch.tensor([2.5], device=G.DEV))
    U = torch.arange(6 * 4, dtype=torch.float32, device=G.DEV).reshape(6, 4).contiguous()
    Y = pasta.ttm(X, U, 2)
    assert pasta.fiber_coords(X, 2)[0].tolist() == [1] and pasta.fiber_coords(X, 2)[1].tolist() == [2]
    assert torch.equal(Y.cpu(), 2.5 * U[3:4].cpu())
    X.close()
    # no stored entries
    E = pasta.CooTensor((4, 5, 6), [torch.zeros(0, dtype=torch.int32, device=G.DEV)] * 3,
                        torch.zeros(0, device=G.DEV))
    assert pasta.fibers(E, 1) == 0
    assert pasta.ttm(E, torch.ones(5, 8, device=G.DEV), 1).shape == (0, 8)
    E.close()
    # other modes wider than the 64-bit key: refused
    big = pasta.CooTensor((1 << 22, 1 << 22, 1 << 22, 2),
                          [torch.tensor([5], dtype=torch.int32, device=G.DEV)] * 3 +
                          [torch.tensor([1], dtype=torch.int32, device=G.DEV)],
                          torch.tensor([1.0], device=G.DEV))
    with pytest.raises(pasta.PastaError) as e:
        pasta.fibers(big, 3)
    assert e.value.name == "PASTA_ERR_UNSUPPORTED"
    assert pasta.fibers(big, 0) == 1  # modes 1, 2, 3: 22 + 22 + 1 bits fit
    big.close()
