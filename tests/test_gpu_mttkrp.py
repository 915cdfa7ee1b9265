"""COO MTTKRP on the GPU vs the FP64 oracle (Eq. (mttkrp-init), Algorithm 6).

Tolerances (rel. Frobenius): 1e-5 for FP32 factors; for BF16/FP16 factors
1e-2 end to end against the FP32 master factors, and 1e-5 for the kernel's
own error against the oracle run on the same rounded factors.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import paper_1902_03317_gb300 as pasta
from paper_1902_03317_gb300 import _lib
from tests import _gpu as G

pytestmark = pytest.mark.gpu

WORKLOADS = [
    # name, nnz, dims, R     (same distributions as the measured shapes, scaled)
    ("uniform3d_200", 20_000, (200, 200, 200), 16),
    ("zipf3d", 200_000, (20_000, 10_000, 4_000), 32),
    ("zipf4d", 200_000, (5_000, 5_000, 500, 100), 64),
    ("cploss3d", 100_000, (2_000, 2_000, 2_000), 32),
    ("zipf5d", 300_000, (8, 100_000, 20_000, 1_000, 100), 16),
]


def check_all_modes(Xh, R, dtype, seed=7, tol=None):
    idx, val = G.host(Xh)
    master, dev, rounded = G.factors(Xh.dims, R, seed, dtype)
    X = G.to_device(Xh)
    for n in range(len(Xh.dims)):
        M = pasta.mttkrp(X, dev, n).cpu().numpy()
        ref_r = oracle.mttkrp(Xh.dims, idx, val, rounded, n, R)
        assert G.rel_err(M, ref_r) < (tol or G.FP32_TOL), f"mode {n} kernel error"
        if dtype != torch.float32 and dtype != torch.float64:
            ref_m = oracle.mttkrp(Xh.dims, idx, val, master, n, R)
            assert G.rel_err(M, ref_m) < G.LOWP_TOL, f"mode {n} end-to-end error"
    X.close()


@pytest.mark.parametrize("name,nnz,dims,R", WORKLOADS)
@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16, torch.float16])
def test_workload_shapes(name, nnz, dims, R, dtype):
    Xh = G.generate(G.small(name, nnz, dims))
    check_all_modes(Xh, R, dtype)


@pytest.mark.parametrize("R", [1, 2, 3, 4, 5, 8, 12, 16, 17, 31, 32, 33, 48, 64, 100, 128, 200, 256])
def test_rank_sweep_fp32(R):
    Xh = G.generate(G.small("zipf3d", 20_000, (3000, 2000, 1000)))
    check_all_modes(Xh, R, torch.float32)


@pytest.mark.parametrize("R", [1, 3, 8, 16, 24, 40, 64, 256])
def test_rank_sweep_bf16(R):
    Xh = G.generate(G.small("zipf4d", 20_000, (800, 800, 80, 20)))
    check_all_modes(Xh, R, torch.bfloat16)


@pytest.mark.parametrize("R", [1, 2, 3, 32, 64, 256])
def test_rank_sweep_fp64(R):
    Xh = G.generate(G.small("zipf3d", 10_000, (900, 500, 300)))
    check_all_modes(Xh, R, torch.float64, tol=1e-12)


@pytest.mark.parametrize("nnz", [0, 1, 2, 3, 4, 5, 31, 33, 511, 512, 513, 2047, 2048, 2049, 16385])
def test_nnz_edges(nnz):
    dims = (40, 30, 20)
    g = torch.Generator().manual_seed(nnz + 1)
    Xh = G.synth.Tensor(None, dims, [torch.randint(0, d, (nnz,), generator=g, dtype=torch.int32) for d in dims],
                        torch.rand(nnz, generator=g) * 2 - 1)
    check_all_modes(Xh, 32, torch.float32)
    check_all_modes(Xh, 16, torch.bfloat16)


def test_single_row_contention():
    # every entry in one output row (mode 0 of size 1) and a very hot row in mode 1
    nnz = 300_000
    g = torch.Generator().manual_seed(3)
    i1 = torch.randint(0, 50, (nnz,), generator=g, dtype=torch.int32)
    i1[: nnz // 2] = 17
    Xh = G.synth.Tensor(None, (1, 50, 400), [torch.zeros(nnz, dtype=torch.int32), i1,
                                             torch.randint(0, 400, (nnz,), generator=g, dtype=torch.int32)],
                        torch.rand(nnz, generator=g))
    check_all_modes(Xh, 32, torch.float32)
    check_all_modes(Xh, 32, torch.bfloat16)


def test_untouched_rows_are_zero_and_output_overwritten():
    dims = (1000, 50, 60)
    nnz = 5000
    g = torch.Generator().manual_seed(4)
    i0 = torch.randint(0, 100, (nnz,), generator=g, dtype=torch.int32) * 7  # rows 0,7,14,... only
    Xh = G.synth.Tensor(None, dims, [i0, torch.randint(0, 50, (nnz,), generator=g, dtype=torch.int32),
                                     torch.randint(0, 60, (nnz,), generator=g, dtype=torch.int32)],
                        torch.rand(nnz, generator=g))
    idx, val = G.host(Xh)
    master, dev, _ = G.factors(dims, 16, 5)
    X = G.to_device(Xh)
    out = torch.full((1000, 16), float("nan"), device=G.DEV)
    M = pasta.mttkrp(X, dev, 0, out=out).cpu().numpy()
    ref = oracle.mttkrp(dims, idx, val, master, 0, 16)
    assert not np.isnan(M).any()
    untouched = np.setdiff1d(np.arange(1000), np.unique(idx[0]))
    assert np.all(M[untouched] == 0)
    assert G.rel_err(M, ref) < G.FP32_TOL
    X.close()


def test_misaligned_factors_take_the_scalar_path():
    Xh = G.generate(G.small("zipf3d", 30_000, (2000, 1000, 500)))
    idx, val = G.host(Xh)
    master, _, _ = G.factors(Xh.dims, 8, 9)
    # factor views starting one element into their storage: not 16-byte aligned
    dev = []
    for u in master:
        big = torch.zeros(u.size + 1, dtype=torch.float32, device=G.DEV)
        big[1:] = torch.from_numpy(u).reshape(-1).to(G.DEV)
        dev.append(big[1:].view(u.shape))
    X = G.to_device(Xh)
    for n in range(3):
        M = pasta.mttkrp(X, dev, n).cpu().numpy()
        assert G.rel_err(M, oracle.mttkrp(Xh.dims, idx, val, master, n, 8)) < G.FP32_TOL
    X.close()


def test_mode_factor_is_not_read():
    Xh = G.generate(G.small("zipf3d", 10_000, (500, 400, 300)))
    idx, val = G.host(Xh)
    master, dev, _ = G.factors(Xh.dims, 16, 2)
    X = G.to_device(Xh)
    for n in range(3):
        Us = list(dev)
        Us[n] = None
        M = pasta.mttkrp(X, Us, n).cpu().numpy()
        assert G.rel_err(M, oracle.mttkrp(Xh.dims, idx, val, master, n, 16)) < G.FP32_TOL
    X.close()


def test_error_statuses():
    dims = (10, 10, 10)
    nnz = 100
    g = torch.Generator().manual_seed(1)
    idx = [torch.randint(0, 10, (nnz,), generator=g, dtype=torch.int32) for _ in dims]
    val = torch.rand(nnz, generator=g)
    bad = [i.clone() for i in idx]
    bad[2][17] = 10
    with pytest.raises(pasta.PastaError) as e:
        pasta.CooTensor(dims, [i.to(G.DEV) for i in bad], val.to(G.DEV))
    assert e.value.name == "PASTA_ERR_INDEX_OOB"
    vbad = val.clone()
    vbad[3] = float("inf")
    with pytest.raises(pasta.PastaError) as e:
        pasta.CooTensor(dims, [i.to(G.DEV) for i in idx], vbad.to(G.DEV))
    assert e.value.name == "PASTA_ERR_NONFINITE"
    X = pasta.CooTensor(dims, [i.to(G.DEV) for i in idx], val.to(G.DEV))
    U = [torch.ones((10, 16), device=G.DEV) for _ in dims]
    M = torch.empty((10, 16), device=G.DEV)
    lib = _lib.lib()
    st = lib.pasta_mttkrp(X.handle, _lib.ptr_array([u.data_ptr() for u in U]), 0, 1, 16,
                          M.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert _lib.STATUS[st] == "PASTA_ERR_NOT_SORTED"
    st = lib.pasta_mttkrp(X.handle, _lib.ptr_array([u.data_ptr() for u in U]), 0, 0, 0,
                          M.data_ptr(), None)
    assert _lib.STATUS[st] == "PASTA_ERR_INVALID_ARG"
    st = lib.pasta_mttkrp(X.handle, _lib.ptr_array([u.data_ptr() for u in U]), 0, 3, 16,
                          M.data_ptr(), None)
    assert _lib.STATUS[st] == "PASTA_ERR_INVALID_ARG"
    X.close()


def test_info_roundtrip():
    Xh = G.generate(G.small("zipf4d", 5000, (100, 90, 80, 7)))
    X = G.to_device(Xh)
    order = ctypes.c_int()
    nnz = ctypes.c_uint64()
    dims = (ctypes.c_uint64 * 8)()
    assert _lib.lib().pasta_coo_info(X.handle, ctypes.byref(order), dims, ctypes.byref(nnz)) == 0
    assert order.value == 4 and nnz.value == 5000 and list(dims)[:4] == [100, 90, 80, 7]
    X.close()
