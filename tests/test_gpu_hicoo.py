"""HiCOO copy (pasta_coo_hicoo) and its MTTKRP (pasta_hicoo_mttkrp) on the
GPU against the oracle.

The copy is integer work: bptr, binds, einds and the values in their order
must equal oracle.hicoo bit for bit (including a case whose key is cut at 64
bits, where ties keep creation order).  The MTTKRP must match the FP64
oracle's MTTKRP of the original COO tensor at 1e-5 (FP32 factors) and, for
BF16, 1e-5 against the oracle on the same rounded factors and 1e-2 end to
end; also with the grid capped so each lane group walks many tiles.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1902_03317_gb300 as pasta
from tests import _gpu as G

pytestmark = pytest.mark.gpu

SHAPES = [
    ("uniform3d_200", 20_000, (200, 200, 200), 16, 3),
    ("zipf3d", 150_000, (20_000, 10_000, 4_000), 32, 7),
    ("zipf4d", 200_000, (5_000, 5_000, 500, 100), 64, 7),
    ("zipf5d", 250_000, (8, 100_000, 20_000, 1_000, 100), 16, 8),
    ("zipf4d", 100_000, (800, 800, 80, 20), 8, 2),
]


def _check_format(X, Xh, bits):
    idx, val = G.host(Xh)
    nb = pasta.hicoo(X, bits)
    bptr, binds, einds, v, _ = oracle.hicoo(Xh.dims, idx, val, bits)
    assert nb == len(bptr) - 1
    gb, gbi, gei, gv = pasta.hicoo_copy_out(X, nb)
    assert np.array_equal(gb.cpu().numpy().astype(np.int64), bptr)
    for k in range(len(Xh.dims)):
        assert np.array_equal(gbi[k].cpu().numpy().astype(np.int64), binds[k]), k
        assert np.array_equal(gei[k].cpu().numpy(), einds[k]), k
    assert np.array_equal(gv.cpu().numpy(), v.astype(np.float32))


@pytest.mark.parametrize("name,nnz,dims,R,bits", SHAPES)
def test_format_matches_oracle(name, nnz, dims, R, bits):
    Xh = G.generate(G.small(name, nnz, dims))
    X = G.to_device(Xh)
    _check_format(X, Xh, bits)
    X.close()


def test_format_with_key_cut_and_rebuild():
    # 2^22-sized modes, 1-bit blocks: 63 block bits, one offset bit kept
    g = torch.Generator().manual_seed(9)
    nnz = 50_000
    dims = (1 << 22, 1 << 22, 1 << 22)
    base = [torch.randint(0, 64, (nnz,), generator=g, dtype=torch.int32) * 1024 for _ in dims]
    idx = [b + torch.randint(0, 4, (nnz,), generator=g, dtype=torch.int32) for b in base]
    Xh = G.synth.Tensor(None, dims, idx, torch.rand(nnz, generator=g))
    X = G.to_device(Xh)
    _check_format(X, Xh, 1)
    _check_format(X, Xh, 5)  # another block size rebuilds the copy
    X.close()


@pytest.mark.parametrize("name,nnz,dims,R,bits", SHAPES)
@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
def test_mttkrp_matches_oracle(name, nnz, dims, R, bits, dtype):
    Xh = G.generate(G.small(name, nnz, dims))
    idx, val = G.host(Xh)
    master, dev, rounded = G.factors(dims, R, 51, dtype)
    X = G.to_device(Xh)
    pasta.hicoo(X, bits)
    for cap in (0, 2):
        with pasta.grid_cap(cap):
            for n in range(len(dims)):
                M = pasta.hicoo_mttkrp(X, dev, n).cpu().numpy()
                assert G.rel_err(M, oracle.mttkrp(dims, idx, val, rounded, n, R)) < G.FP32_TOL, (n, cap)
                if dtype != torch.float32:
                    assert G.rel_err(M, oracle.mttkrp(dims, idx, val, master, n, R)) < G.LOWP_TOL, n
    X.close()


@pytest.mark.parametrize("nnz", [0, 1, 3, 5, 511, 512, 513, 4097])
def test_small_and_ragged(nnz):
    dims = (40, 30, 20)
    g = torch.Generator().manual_seed(nnz + 7)
    Xh = G.synth.Tensor(None, dims, [torch.randint(0, d, (nnz,), generator=g, dtype=torch.int32) for d in dims],
                        torch.rand(nnz, generator=g) * 2 - 1)
    idx, val = G.host(Xh)
    master, dev, _ = G.factors(dims, 32, 52)
    X = G.to_device(Xh)
    _check_format(X, Xh, 3)
    for n in range(3):
        out = torch.full((dims[n], 32), float("nan"), device=G.DEV)
        M = pasta.hicoo_mttkrp(X, dev, n, out=out).cpu().numpy()
        assert not np.isnan(M).any()
        assert G.rel_err(M, oracle.mttkrp(dims, idx, val, master, n, 32)) < G.FP32_TOL, n
    X.close()


def test_errors():
    Xh = G.generate(G.small("zipf3d", 2000, (100, 90, 80)))
    X = G.to_device(Xh)
    _, dev, _ = G.factors((100, 90, 80), 32, 53)
    with pytest.raises(pasta.PastaError) as e:
        pasta.hicoo_mttkrp(X, dev, 0)
    assert e.value.name == "PASTA_ERR_NOT_SORTED"
    with pytest.raises(pasta.PastaError) as e:
        pasta.hicoo(X, 9)
    assert e.value.name == "PASTA_ERR_INVALID_ARG"
    pasta.hicoo(X, 4)
    _, dev5, _ = G.factors((100, 90, 80), 5, 54)
    with pytest.raises(pasta.PastaError) as e:
        pasta.hicoo_mttkrp(X, dev5, 1)
    assert e.value.name == "PASTA_ERR_UNSUPPORTED"
    X.close()


@pytest.mark.parametrize("dtype,R", [(torch.float32, 4), (torch.float32, 8), (torch.float32, 128),
                                     (torch.bfloat16, 8), (torch.bfloat16, 256), (torch.float16, 32)])
def test_rank_and_type_sweep(dtype, R):
    """The lane-group geometry from 1 lane per row (FP32 R = 4) to 32 (BF16
    R = 256), and FP16 factors."""
    Xh = G.generate(G.small("zipf4d", 30_000, (900, 800, 70, 20)))
    idx, val = G.host(Xh)
    master, dev, rounded = G.factors(Xh.dims, R, 55, dtype)
    X = G.to_device(Xh)
    pasta.hicoo(X, 4)
    for n in range(4):
        M = pasta.hicoo_mttkrp(X, dev, n).cpu().numpy()
        assert G.rel_err(M, oracle.mttkrp(Xh.dims, idx, val, rounded, n, R)) < G.FP32_TOL, n
    X.close()


def test_contended_rows_stay_within_the_fp32_bar():
    """A short, heavily shared output mode (zipf5d's 8-row mode 0: 500k
    entries per row, partials from about a thousand tiles each) and the mode
    last in the in-block order (a new row almost every entry): the FP64
    image keeps HiCOO's MTTKRP within 1e-5 of the FP64 oracle."""
    dims = (8, 400_000, 100_000, 10_000, 1_000)
    Xh = G.generate(G.small("zipf5d", 4_000_000, dims))
    idx, val = G.host(Xh)
    X = G.to_device(Xh)
    master, dev, _ = G.factors(dims, 16, 13)
    pasta.hicoo(X, 8)
    for mode in (0, 4):
        ref = oracle.mttkrp(dims, idx, val, master, mode)
        H = pasta.hicoo_mttkrp(X, dev, mode)
        assert G.rel_err(H.cpu().numpy(), ref) < G.FP32_TOL, mode
    X.close()
