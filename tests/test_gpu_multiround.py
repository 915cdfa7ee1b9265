"""The kernels' multi-round path (block tiles walked in turn by a grid smaller
than the stream) against the FP64 oracle, element by element.

The streaming kernels stride over block tiles (``bt += gridDim.x``).  A
block's second and later tiles reuse the shared-memory words that served as
its end-of-tile slots, carry no register state from the previous tile, and
start with the open-run test against the entry before the tile.  With the full
grid this path only runs above about ten million entries, so two sets of
cases cover it:

* the parity shapes of the other files with ``pasta.grid_cap`` limiting every
  launch to 1-3 blocks, so each block walks four or more block tiles;
* one 16M-entry tensor with zipf3d's distributions at the full launch
  configuration (two rounds of the resident grid), every output row of every
  mode of MTTKRP and of the fused loss and gradients compared with the oracle.

Tolerances as elsewhere: 1e-5 rel. Frobenius for FP32 factors; for BF16 the
kernel error against the oracle on the same rounded factors (1e-5) and the
end-to-end error against the FP32 master factors (1e-2).
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1902_03317_gb300 as pasta
from tests import _gpu as G

pytestmark = pytest.mark.gpu

SHAPES = [
    # name, nnz, dims, R, grid cap
    ("zipf3d", 200_000, (20_000, 10_000, 4_000), 32, 2),
    ("zipf4d", 200_000, (5_000, 5_000, 500, 100), 64, 3),
    ("cploss3d", 100_000, (2_000, 2_000, 2_000), 32, 1),
    ("zipf5d", 300_000, (8, 100_000, 20_000, 1_000, 100), 16, 2),
]


def _block_tiles(nnz, R, esize):
    """Block tiles of the streaming kernels at the longest group tile: 8 warps
    x (32 / L) lane groups x 512 entries, L = R * esize / 16 lanes per row."""
    L = R * esize // 16
    return -(-nnz // (8 * (32 // L) * max(512, 4 * L)))


def _rounds_cap(nnz, R, dtype, cap):
    """The largest cap <= ``cap`` that leaves every block four or more block
    tiles to walk."""
    tiles = _block_tiles(nnz, R, 4 if dtype == torch.float32 else 2)
    cap = max(1, min(cap, tiles // 4))
    assert tiles >= 4 * cap
    return cap


@pytest.mark.parametrize("name,nnz,dims,R,cap", SHAPES)
@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
def test_mttkrp_multi_round(name, nnz, dims, R, cap, dtype):
    cap = _rounds_cap(nnz, R, dtype, cap)
    Xh = G.generate(G.small(name, nnz, dims))
    idx, val = G.host(Xh)
    master, dev, rounded = G.factors(dims, R, 31, dtype)
    X = G.to_device(Xh)
    with pasta.grid_cap(cap):
        for n in range(len(dims)):
            M = pasta.mttkrp(X, dev, n).cpu().numpy()
            assert G.rel_err(M, oracle.mttkrp(dims, idx, val, rounded, n, R)) < G.FP32_TOL, n
            if dtype != torch.float32:
                assert G.rel_err(M, oracle.mttkrp(dims, idx, val, master, n, R)) < G.LOWP_TOL, n
    assert pasta.api._lib.lib().pasta_get_grid_cap() == 0
    X.close()


@pytest.mark.parametrize("name,nnz,dims,R,cap", SHAPES)
@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
def test_loss_and_gradients_multi_round(name, nnz, dims, R, cap, dtype):
    cap = _rounds_cap(nnz, R, dtype, cap)
    Xh = G.generate(G.small(name, nnz, dims))
    idx, val = G.host(Xh)
    _, dev, rounded = G.factors(dims, R, 32, dtype)
    X = G.to_device(Xh)
    for k in range(len(dims)):
        X.sort_by_mode(k)
    ref_loss, ref_e = oracle.cp_loss(dims, idx, val, rounded, want_resid=True)
    ref_G = oracle.cp_grad(dims, idx, val, rounded, g=0.75)
    gs = torch.tensor(0.75, dtype=torch.float64, device=G.DEV)
    with pasta.grid_cap(cap):
        # fused loss + every gradient (one pass per mode, the first also summing the loss)
        loss, grads = pasta.cp_loss_fwd_bwd(X, dev, gscale=gs)
        assert abs(loss.item() - ref_loss) <= G.FP32_TOL * ref_loss
        for k in range(len(dims)):
            assert G.rel_err(grads[k].cpu().numpy(), ref_G[k]) < G.FP32_TOL, k
        # forward alone, with residuals, over the creation-order and a sorted copy
        for mode in (-1, len(dims) - 1):
            loss, e = pasta.cp_loss_fwd(X, dev, mode, want_resid=True)
            assert abs(loss.item() - ref_loss) <= G.FP32_TOL * ref_loss, mode
            perm = np.arange(nnz) if mode < 0 else X.copy_out(mode)[2].cpu().numpy().astype(np.int64)
            assert G.rel_err(e.cpu().numpy(), ref_e[perm]) < G.FP32_TOL, mode
        # per-mode backward without the loss
        grads = pasta.cp_loss_bwd(X, dev, pasta.api.BWD_PER_MODE, gscale=gs)
        for k in range(len(dims)):
            assert G.rel_err(grads[k].cpu().numpy(), ref_G[k]) < G.FP32_TOL, k
    X.close()


@pytest.mark.parametrize("dtype,R", [(torch.float64, 32), (torch.float32, 5)])
def test_general_kernels_multi_round(dtype, R):
    """FP64 factors and R = 5 take the general (non-streaming) kernels, which
    stride over warp tiles the same way."""
    nnz, dims = 120_000, (3_000, 2_000, 1_000)
    Xh = G.generate(G.small("zipf3d", nnz, dims))
    idx, val = G.host(Xh)
    master, dev, rounded = G.factors(dims, R, 33, dtype)
    X = G.to_device(Xh)
    for k in range(3):
        X.sort_by_mode(k)
    tol = 1e-12 if dtype == torch.float64 else G.FP32_TOL
    ref_loss = oracle.cp_loss(dims, idx, val, rounded)
    ref_G = oracle.cp_grad(dims, idx, val, rounded)
    with pasta.grid_cap(1):
        for n in range(3):
            M = pasta.mttkrp(X, dev, n).cpu().numpy()
            assert G.rel_err(M, oracle.mttkrp(dims, idx, val, rounded, n, R)) < tol, n
        loss, grads = pasta.cp_loss_fwd_bwd(X, dev)
        assert abs(loss.item() - ref_loss) <= tol * ref_loss
        for k in range(3):
            assert G.rel_err(grads[k].cpu().numpy(), ref_G[k]) < tol, k
        for mode in (-1, 0):  # one-pass forms: atomics for the other modes
            grads = pasta.cp_loss_bwd(X, dev, mode)
            for k in range(3):
                assert G.rel_err(grads[k].cpu().numpy(), ref_G[k]) < tol, (mode, k)
    X.close()


def test_grid_cap_rejects_negative():
    with pytest.raises(pasta.PastaError):
        with pasta.grid_cap(-1):
            pass
    assert pasta.api._lib.lib().pasta_get_grid_cap() == 0


@pytest.mark.fullsize
def test_zipf3d_16m_every_row():
    """16M entries with zipf3d's dims and distributions, R = 32 FP32, the
    launch configuration of the bench (no cap): two rounds of the resident
    grid.  Every row of every mode of MTTKRP, the loss and every row of every
    gradient against the oracle; then MTTKRP again with the grid capped to
    one block per SM (seven rounds)."""
    nnz = 16_000_000
    dims = (1_000_000, 500_000, 200_000)
    Xh = G.generate(G.small("zipf3d", nnz, dims), device=G.DEV).to("cpu")
    idx, val = G.host(Xh)
    master, dev, _ = G.factors(dims, 32, 34)
    X = G.to_device(Xh)
    for k in range(3):
        X.sort_by_mode(k)
    assert _block_tiles(nnz, 32, 4) > 152 * 4  # more block tiles than the resident grid (4 blocks/SM)
    refs = [oracle.mttkrp(dims, idx, val, master, n, 32) for n in range(3)]
    for n in range(3):
        M = pasta.mttkrp(X, dev, n).cpu().numpy()
        assert G.rel_err(M, refs[n]) < G.FP32_TOL, n
        touched = np.unique(idx[n])
        assert np.all(M[np.setdiff1d(np.arange(dims[n]), touched)] == 0), n
    with pasta.grid_cap(152):
        for n in range(3):
            M = pasta.mttkrp(X, dev, n).cpu().numpy()
            assert G.rel_err(M, refs[n]) < G.FP32_TOL, n
    del refs
    ref_loss = oracle.cp_loss(dims, idx, val, master)
    ref_G = oracle.cp_grad(dims, idx, val, master)
    loss, grads = pasta.cp_loss_fwd_bwd(X, dev)
    assert abs(loss.item() - ref_loss) <= G.FP32_TOL * ref_loss
    for k in range(3):
        assert G.rel_err(grads[k].cpu().numpy(), ref_G[k]) < G.FP32_TOL, k
    X.close()
