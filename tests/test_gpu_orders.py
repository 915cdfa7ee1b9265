"""Every operation at the orders the streaming kernels do not cover (2 for the
loss kinds, 6-8 for all) against the FP64 oracle: MTTKRP on every mode, the
loss with every gradient, one CP-ALS sweep, TTM and TTV.  Tolerances as in
the per-operation test files (MTTKRP bar 1e-5; CP-ALS 1e-4 / 1e-5)."""
import numpy as np
import pytest
import torch

import oracle
import paper_1902_03317_gb300 as pasta
from tests import _gpu as G

pytestmark = pytest.mark.gpu

DIMS = {2: (300, 200), 6: (9, 8, 10, 11, 8, 9), 7: (8, 9, 8, 10, 9, 8, 11), 8: (8, 9, 10, 8, 9, 11, 8, 10)}


def _tensor(order, nnz=4000, seed=0):
    g = np.random.default_rng(seed + order)
    dims = DIMS[order]
    idx = [g.integers(0, d, nnz).astype(np.uint32) for d in dims]
    val = g.uniform(-1, 1, nnz)
    X = pasta.CooTensor(dims, [torch.tensor(ix.astype(np.int32), device=G.DEV) for ix in idx],
                        torch.tensor(val, dtype=torch.float32, device=G.DEV))
    return dims, idx, val.astype(np.float32).astype(np.float64), X


@pytest.mark.parametrize("order", [2, 6, 7, 8])
def test_mttkrp_and_loss(order):
    dims, idx, val, X = _tensor(order)
    for R in (8, 5):
        g = torch.Generator().manual_seed(R)
        Us = [torch.randn(d, R, generator=g) for d in dims]
        Ud = [u.to(G.DEV) for u in Us]
        Uh = [u.double().numpy() for u in Us]
        for n in range(order):
            M = pasta.mttkrp(X, Ud, n)
            assert G.rel_err(M.cpu().numpy(), oracle.mttkrp(dims, idx, val, Uh, n)) < G.FP32_TOL, (order, R, n)
        loss, grads = pasta.cp_loss_fwd_bwd(X, Ud)
        ref = oracle.cp_loss(dims, idx, val, Uh)
        assert abs(float(loss) - ref) <= 1e-5 * abs(ref), (order, R, float(loss), ref)
        ref_g = oracle.cp_grad(dims, idx, val, Uh)
        for k in range(order):
            assert G.rel_err(grads[k].cpu().numpy(), ref_g[k]) < G.FP32_TOL, (order, R, k)
    X.close()


@pytest.mark.parametrize("order", [2, 6, 8])
def test_als_ttm_ttv(order):
    dims, idx, val, X = _tensor(order, nnz=6000)
    R = 3
    g = torch.Generator().manual_seed(11)
    Us = [torch.randn(d, R, generator=g) for d in dims]
    Ud = [u.to(G.DEV).contiguous() for u in Us]
    lam, fit = pasta.cp_als_sweep(X, Ud)
    Ur, lam_r, fit_r = oracle.cp_als_sweep(dims, idx, val, [u.double().numpy() for u in Us])
    for k in range(order):
        assert G.rel_err(Ud[k].cpu().numpy(), Ur[k]) < 1e-4, (order, k)
    assert abs(float(fit) - fit_r) < 1e-5
    for n in (0, order - 1):
        U = torch.randn(dims[n], 8, device=G.DEV)
        Y = pasta.ttm(X, U, n)
        coords, ref = oracle.ttm(dims, idx, val, U.double().cpu().numpy(), n)
        for a, b in zip(pasta.fiber_coords(X, n), coords):
            assert np.array_equal(a.cpu().numpy().astype(np.uint32), b)
        assert G.rel_err(Y.cpu().numpy(), ref) < G.FP32_TOL
        v = torch.randn(dims[n], device=G.DEV)
        y = pasta.ttv(X, v, n)
        assert G.rel_err(y.cpu().numpy(), oracle.ttv(dims, idx, val, v.double().cpu().numpy(), n)[1]) < G.FP32_TOL
    X.close()
