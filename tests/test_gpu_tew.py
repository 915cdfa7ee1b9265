"""TEW-eq and TS (pasta_tew_eq, pasta_ts) on the GPU vs the FP64 oracle.

Coordinates must come back bit-exact.  Values: the GPU computes each value
with one IEEE FP32 operation, i.e. the exact result of the operation on the
FP32 inputs rounded once; the oracle computes it in FP64 and is rounded to
FP32 here.  The FP64 result is exact for products of FP32 numbers and for
most sums, so the two agree except where rounding twice (FP64, then FP32)
lands one unit in the last place away: the bar is at most 1 ulp, and
multiplication must be bit-exact.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1902_03317_gb300 as pasta
from paper_1902_03317_gb300 import synth
from tests import _gpu as G

pytestmark = pytest.mark.gpu


def ulp_distance(got: np.ndarray, ref64: np.ndarray) -> np.ndarray:
    a = np.asarray(got, dtype=np.float32).view(np.int32).astype(np.int64)
    b = np.asarray(ref64, dtype=np.float64).astype(np.float32).view(np.int32).astype(np.int64)
    # map the sign-magnitude bit patterns onto a monotone integer line
    a = np.where(a < 0, -(a & 0x7FFFFFFF), a)
    b = np.where(b < 0, -(b & 0x7FFFFFFF), b)
    return np.abs(a - b)


def _pair(nnz, dims, seed=5):
    wl = G.small("zipf3d", nnz, dims, seed=seed)
    Xh = synth.generate(wl)
    idx, vx = G.host(Xh)
    g = torch.Generator().manual_seed(seed + 1)
    vy = (torch.rand(nnz, generator=g) * 1.5 + 0.5) * torch.where(torch.rand(nnz, generator=g) < 0.5, -1.0, 1.0)
    X = G.to_device(Xh)
    Y = pasta.CooTensor(Xh.dims, [i.to(G.DEV) for i in Xh.idx], vy.to(torch.float32).to(G.DEV))
    return wl, X, Y, idx, vx, vy.to(torch.float32).double().numpy()


@pytest.mark.parametrize("nnz,dims", [(300_001, (5_000, 3_000, 2_000)), (1, (3, 3, 3)), (0, (3, 3, 3))])
@pytest.mark.parametrize("op", oracle.OPS)
def test_tew_eq_matches_oracle(nnz, dims, op):
    if nnz == 0:
        X = pasta.CooTensor(dims, [torch.zeros(0, dtype=torch.int32, device=G.DEV)] * 3,
                            torch.zeros(0, device=G.DEV))
        Z = pasta.tew_eq(X, X, op)
        assert Z.nnz == 0
        return
    wl, X, Y, idx, vx, vy = _pair(nnz, dims)
    Z = pasta.tew_eq(X, Y, op)
    zi, zv, _ = Z.copy_out()
    for k in range(3):
        assert np.array_equal(zi[k].cpu().numpy().astype(np.uint32), idx[k])
    _, ref = oracle.tew_eq(idx, vx, idx, vy, op)
    d = ulp_distance(zv.cpu().numpy(), ref)
    assert d.max() <= (0 if op == "mul" else 1), (op, int(d.max()))


@pytest.mark.parametrize("op", oracle.OPS)
@pytest.mark.parametrize("s", [-1.75, 3.3])
def test_ts_matches_oracle(op, s):
    wl, X, Y, idx, vx, vy = _pair(200_003, (4_000, 2_000, 1_000))
    Z = pasta.ts(X, op, s)
    zi, zv, _ = Z.copy_out()
    for k in range(3):
        assert np.array_equal(zi[k].cpu().numpy().astype(np.uint32), idx[k])
    _, ref = oracle.ts(idx, vx, op, float(np.float32(s)))  # the scalar is rounded to FP32 once
    d = ulp_distance(zv.cpu().numpy(), ref)
    assert d.max() <= (0 if op == "mul" else 1), (op, s, int(d.max()))


def test_output_handle_is_reused_and_derived_data_dropped():
    wl, X, Y, idx, vx, vy = _pair(50_000, (500, 400, 300))
    out = pasta.ts(X, "mul", 2.0)
    out.sort_by_mode(0)
    Z = pasta.tew_eq(X, Y, "add", out=out)
    assert Z is out
    _, zv, _ = Z.copy_out()
    assert ulp_distance(zv.cpu().numpy(), vx + vy).max() <= 1
    # the sorted copy was dropped: MTTKRP needs a new sort, which then agrees
    Us = [torch.randn(d, 8, device=G.DEV) for d in wl.dims]
    M = pasta.mttkrp(Z, Us, 0)
    ref = oracle.mttkrp(wl.dims, idx, zv.cpu().double().numpy(), [u.cpu().double().numpy() for u in Us], 0)
    assert G.rel_err(M.cpu().numpy(), ref) < G.FP32_TOL
    with pytest.raises(ValueError):
        pasta.ts(X, "add", 1.0, out=X)


def test_tew_eq_rejects_other_coordinates_and_shapes():
    wl, X, Y, idx, vx, vy = _pair(10_000, (300, 200, 100))
    moved = [torch.tensor(ix.astype(np.int32)) for ix in idx]
    moved[2][17] = (moved[2][17] + 1) % 100
    W = pasta.CooTensor(wl.dims, [m.to(G.DEV) for m in moved], torch.tensor(vy, dtype=torch.float32, device=G.DEV))
    with pytest.raises(pasta.PastaError) as e:
        pasta.tew_eq(X, W, "add")
    assert e.value.name == "PASTA_ERR_INVALID_ARG"
    V = pasta.CooTensor((300, 200, 101), [torch.tensor(ix.astype(np.int32), device=G.DEV) for ix in idx],
                        torch.tensor(vy, dtype=torch.float32, device=G.DEV))
    with pytest.raises(pasta.PastaError):
        pasta.tew_eq(X, V, "mul")
