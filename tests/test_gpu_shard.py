"""Range forms for splitting a tensor over ranks (pasta_mttkrp_range,
pasta_cp_loss_fwd_bwd_range), run one range after another on one GPU: the
outputs of ranges that partition the stored entries (shard.aligned_ranges,
the cuts bench.py's sharded step uses) must sum to the whole tensor's, and
match the FP64 oracle at 1e-5 (FP32 factors).  No collective and no second
GPU are involved; the cross-rank completion of range-end rows is covered by
the gloo tests."""
import numpy as np
import pytest
import torch

import oracle
import paper_1902_03317_gb300 as pasta
from paper_1902_03317_gb300 import shard
from tests import _gpu as G

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name,nnz,dims,R", [
    ("zipf3d", 200_003, (20_000, 10_000, 4_000), 32),
    ("zipf5d", 150_001, (8, 50_000, 10_000, 1_000, 100), 16),
    ("zipf3d", 30_001, (900, 500, 300), 5),  # general kernels
])
@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_ranges_sum_to_whole(name, nnz, dims, R, world):
    Xh = G.generate(G.small(name, nnz, dims))
    idx, val = G.host(Xh)
    master, dev, _ = G.factors(dims, R, 61)
    X = G.to_device(Xh)
    X.sort_all()
    ranges = shard.aligned_ranges(nnz, world)
    for n in range(len(dims)):
        tot = torch.zeros((dims[n], R), dtype=torch.float64, device=G.DEV)
        for lo, hi in ranges:
            tot += pasta.mttkrp_range(X, dev, n, lo, hi).double()
        assert G.rel_err(tot.cpu().numpy(), oracle.mttkrp(dims, idx, val, master, n, R)) < G.FP32_TOL, n
    loss = 0.0
    grads = [torch.zeros((d, R), dtype=torch.float64, device=G.DEV) for d in dims]
    gs = torch.tensor(0.5, dtype=torch.float64, device=G.DEV)
    for lo, hi in ranges:
        l, gk = pasta.cp_loss_fwd_bwd_range(X, dev, lo, hi, gscale=gs)
        loss += float(l)
        for k in range(len(dims)):
            grads[k] += gk[k].double()
    ref_loss = oracle.cp_loss(dims, idx, val, master)
    ref_G = oracle.cp_grad(dims, idx, val, master, g=0.5)
    assert abs(loss - ref_loss) <= G.FP32_TOL * ref_loss
    for k in range(len(dims)):
        assert G.rel_err(grads[k].cpu().numpy(), ref_G[k]) < G.FP32_TOL, k
    X.close()


def test_range_errors():
    Xh = G.generate(G.small("zipf3d", 1000, (100, 90, 80)))
    X = G.to_device(Xh)
    _, dev, _ = G.factors((100, 90, 80), 16, 62)
    with pytest.raises(pasta.PastaError) as e:
        pasta.mttkrp_range(X, dev, 0, 2, 10)
    assert e.value.name == "PASTA_ERR_ALIGNMENT"
    with pytest.raises(pasta.PastaError) as e:
        pasta.mttkrp_range(X, dev, 0, 0, 1001)
    assert e.value.name == "PASTA_ERR_INVALID_ARG"
    M = pasta.mttkrp_range(X, dev, 1, 8, 8)  # an empty range: all zeros
    assert float(M.abs().sum()) == 0.0
    X.close()
