"""Sparse CP loss forward/backward on the GPU vs the FP64 oracle.

loss = 1/2 sum_m (x_m - sum_r prod_k U_k(i_k(m), r))^2 over stored entries;
its gradient is -(mode-k MTTKRP of the residual tensor) for every mode k.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1902_03317_gb300 as pasta
from tests import _gpu as G

pytestmark = pytest.mark.gpu

SHAPES = [
    ("uniform3d_200", 20_000, (200, 200, 200), 16),
    ("zipf3d", 100_000, (10_000, 5_000, 2_000), 32),
    ("zipf4d", 100_000, (3_000, 3_000, 300, 60), 64),
    ("cploss3d", 100_000, (3_000, 3_000, 3_000), 32),
    ("zipf5d", 100_000, (8, 50_000, 10_000, 1_000, 100), 16),
]


def _copy_order(X, mode, nnz):
    if mode < 0:
        return np.arange(nnz)
    X.sort_by_mode(mode)
    return X.copy_out(mode)[2].cpu().numpy().astype(np.int64)


@pytest.mark.parametrize("name,nnz,dims,R", SHAPES)
def test_loss_and_grad_fp32(name, nnz, dims, R):
    Xh = G.generate(G.small(name, nnz, dims))
    idx, val = G.host(Xh)
    master, dev, _ = G.factors(dims, R, 11)
    X = G.to_device(Xh)
    ref_loss, ref_e = oracle.cp_loss(dims, idx, val, master, want_resid=True)
    ref_G = oracle.cp_grad(dims, idx, val, master, g=1.5)
    gs = torch.tensor(1.5, dtype=torch.float64, device=G.DEV)
    for mode in [-1] + list(range(len(dims))) + [-2]:
        fmode = 0 if mode == -2 else mode
        loss, e = pasta.cp_loss_fwd(X, dev, fmode, want_resid=True)
        assert abs(loss.item() - ref_loss) <= G.FP32_TOL * ref_loss
        perm = _copy_order(X, fmode, nnz)
        assert G.rel_err(e.cpu().numpy(), ref_e[perm]) < G.FP32_TOL
        grads = pasta.cp_loss_bwd(X, dev, mode, gscale=gs)
        for k in range(len(dims)):
            assert G.rel_err(grads[k].cpu().numpy(), ref_G[k]) < G.FP32_TOL, (mode, k)
    X.close()


@pytest.mark.parametrize("dtype", [torch.bfloat16, torch.float16])
@pytest.mark.parametrize("name,nnz,dims,R", [SHAPES[1], SHAPES[3], SHAPES[4]])
def test_loss_and_grad_low_precision(name, nnz, dims, R, dtype):
    Xh = G.generate(G.small(name, nnz, dims))
    idx, val = G.host(Xh)
    master, dev, rounded = G.factors(dims, R, 12, dtype)
    X = G.to_device(Xh)
    X.sort_by_mode(0)
    loss = pasta.cp_loss_fwd(X, dev, 0).item()
    grads = pasta.cp_loss_bwd(X, dev, 0)
    grads_pm = pasta.cp_loss_bwd(X, dev, -2)
    # kernel error: against the oracle on the same rounded factors
    ref_loss_r = oracle.cp_loss(dims, idx, val, rounded)
    assert abs(loss - ref_loss_r) <= G.FP32_TOL * ref_loss_r
    ref_G_r = oracle.cp_grad(dims, idx, val, rounded)
    # end-to-end error: against the FP32 master factors
    ref_loss_m = oracle.cp_loss(dims, idx, val, master)
    assert abs(loss - ref_loss_m) <= G.LOWP_TOL * ref_loss_m
    ref_G_m = oracle.cp_grad(dims, idx, val, master)
    for k in range(len(dims)):
        for g in (grads[k].cpu().numpy(), grads_pm[k].cpu().numpy()):
            assert G.rel_err(g, ref_G_r[k]) < G.FP32_TOL
            assert G.rel_err(g, ref_G_m[k]) < G.LOWP_TOL
    X.close()


def test_loss_is_bitwise_reproducible():
    Xh = G.generate(G.small("zipf3d", 200_000, (20_000, 10_000, 4_000)))
    _, dev, _ = G.factors(Xh.dims, 32, 3)
    X = G.to_device(Xh)
    a = pasta.cp_loss_fwd(X, dev).item()
    b = pasta.cp_loss_fwd(X, dev).item()
    assert a == b
    X.close()


def test_planted_model_loss_is_noise_level():
    """Values = planted rank-16 model + N(0, 0.01^2); fitting with
    [planted | 0] (R = 32) leaves only the noise: loss ~ nnz * sigma^2 / 2."""
    wl = G.small("cploss3d", 200_000, (5_000, 5_000, 5_000))
    Xh = G.generate(wl)
    idx, val = G.host(Xh)
    fit = [torch.cat([p, torch.zeros_like(p)], dim=1) for p in Xh.planted]
    X = G.to_device(Xh)
    loss = pasta.cp_loss_fwd(X, [f.to(G.DEV).contiguous() for f in fit]).item()
    expect = 0.5 * wl.nnz * wl.noise_sigma ** 2
    assert abs(loss - expect) < 0.02 * expect  # chi-square spread, 200k entries
    ref = oracle.cp_loss(wl.dims, idx, val, [f.numpy() for f in fit])
    # FP32 model values near |model| ~ 4 carry ~1e-6 absolute error each,
    # against residuals of 1e-2: the loss agrees to ~1e-3 relative.
    assert abs(loss - ref) < 2e-3 * ref
    X.close()


def test_autograd_function_matches_kernels_and_returns_param_dtype():
    Xh = G.generate(G.small("zipf4d", 50_000, (2000, 2000, 200, 50)))
    _, dev, _ = G.factors(Xh.dims, 32, 4, torch.bfloat16)
    X = G.to_device(Xh)
    X.sort_by_mode(1)
    params = [u.clone().requires_grad_(True) for u in dev]
    loss = pasta.cp_loss(X, params, 1)
    (3.0 * loss).backward()
    ref = pasta.cp_loss_bwd(X, dev, 1, gscale=torch.tensor(3.0, dtype=torch.float64))
    for p, g in zip(params, ref):
        assert p.grad.dtype == torch.bfloat16
        # the two runs add with atomics in different orders; BF16 rounding
        # (2^-9 relative) dominates the difference
        assert G.rel_err(p.grad.float().cpu().numpy(), g.cpu().numpy()) < 4e-3
    X.close()


def test_gradcheck_fp64_30cube():
    """torch.autograd.gradcheck (FP64 finite differences) on a 30x30x30
    tensor with 500 entries, R = 32, through the FP64 kernels."""
    wl = G.small("cploss3d", 500, (30, 30, 30))
    Xh = G.generate(wl)
    X = G.to_device(Xh)
    Us = [u.to(G.DEV) for u in G.synth.generate_factors(wl.dims, 32, seed=5, dtype=torch.float64)]
    Us = [u.requires_grad_(True) for u in Us]
    # FD noise: the loss is ~1e4 in FP64, so (L(u+h) - L(u-h)) / 2h carries
    # ~1e-16 * 1e4 / 1e-6 = 1e-6 .. 1e-5 absolute error; gradcheck's default
    # atol = 1e-5, rtol = 1e-3 covers it.
    for mode in (-1, 0, -2):
        assert torch.autograd.gradcheck(lambda *u: pasta.cp_loss(X, u, mode), Us, eps=1e-6)
    X.close()


def test_gradient_vs_oracle_finite_differences():
    """FP32 GPU gradient vs central differences of the FP64 oracle loss on a
    sample of entries (h = 1e-6)."""
    wl = G.small("cploss3d", 500, (30, 30, 30))
    Xh = G.generate(wl)
    idx, val = G.host(Xh)
    master, dev, _ = G.factors(wl.dims, 32, 6)
    X = G.to_device(Xh)
    grads = [g.cpu().numpy() for g in pasta.cp_loss_bwd(X, dev)]
    rng = np.random.default_rng(0)
    h = 1e-6
    for _ in range(40):
        k = int(rng.integers(0, 3))
        i = int(rng.choice(idx[k]))
        r = int(rng.integers(0, 32))
        up = [u.astype(np.float64).copy() for u in master]
        um = [u.astype(np.float64).copy() for u in master]
        up[k][i, r] += h
        um[k][i, r] -= h
        fd = (oracle.cp_loss(wl.dims, idx, val, up) - oracle.cp_loss(wl.dims, idx, val, um)) / (2 * h)
        assert abs(grads[k][i, r] - fd) <= 1e-4 * max(1.0, abs(fd))
    X.close()


def test_convert_rounds_to_nearest_even():
    x = torch.randn(100_003, device=G.DEV)
    for dt in (torch.bfloat16, torch.float16, torch.float64):
        y = pasta.convert(x, dt)
        assert torch.equal(y, x.to(dt))
    z = pasta.convert(x.double(), torch.float32)
    assert torch.equal(z, x)


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
@pytest.mark.parametrize("name,nnz,dims,R", [SHAPES[1], SHAPES[2], SHAPES[4]])
def test_fused_loss_and_grad(name, nnz, dims, R, dtype):
    """pasta_cp_loss_fwd_bwd: the loss and all gradients in N passes."""
    Xh = G.generate(G.small(name, nnz, dims))
    idx, val = G.host(Xh)
    _, dev, rounded = G.factors(dims, R, 13, dtype)
    X = G.to_device(Xh)
    loss, grads = pasta.cp_loss_fwd_bwd(X, dev, gscale=torch.tensor(0.5, dtype=torch.float64))
    ref_loss = oracle.cp_loss(dims, idx, val, rounded)
    assert abs(loss.item() - ref_loss) <= G.FP32_TOL * ref_loss
    ref_G = oracle.cp_grad(dims, idx, val, rounded, g=0.5)
    for k in range(len(dims)):
        assert G.rel_err(grads[k].cpu().numpy(), ref_G[k]) < G.FP32_TOL, k
    # reproducible bits
    loss2, _ = pasta.cp_loss_fwd_bwd(X, dev, gscale=torch.tensor(0.5, dtype=torch.float64))
    assert loss2.item() == loss.item()
    X.close()


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
def test_autograd_per_mode_uses_fused_pass_and_scales(dtype):
    Xh = G.generate(G.small("zipf3d", 60_000, (5_000, 3_000, 1_000)))
    idx, val = G.host(Xh)
    _, dev, rounded = G.factors(Xh.dims, 32, 14, dtype)
    X = G.to_device(Xh)
    params = [u.clone().requires_grad_(True) for u in dev]
    loss = pasta.cp_loss(X, params)  # mode -2
    (2.5 * loss).backward(retain_graph=True)
    ref_G = oracle.cp_grad(Xh.dims, idx, val, rounded, g=2.5)
    tol = G.FP32_TOL if dtype == torch.float32 else 4e-3  # BF16 rounding of the gradient
    for p, r in zip(params, ref_G):
        assert p.grad.dtype == dtype
        assert G.rel_err(p.grad.float().cpu().numpy(), r) < tol
    # a second backward recomputes instead of reusing the scaled gradients
    for p in params:
        p.grad = None
    loss.backward()
    ref_1 = oracle.cp_grad(Xh.dims, idx, val, rounded, g=1.0)
    for p, r in zip(params, ref_1):
        assert G.rel_err(p.grad.float().cpu().numpy(), r) < tol
    X.close()


def test_convert_scaled():
    x = torch.randn(10_001, device=G.DEV)
    sc = torch.tensor(-1.75, dtype=torch.float64, device=G.DEV)
    assert torch.equal(pasta.convert(x, torch.float32, scale=sc), x * -1.75)
    assert torch.equal(pasta.convert(x, torch.bfloat16, scale=sc), (x * -1.75).to(torch.bfloat16))
    y = x.clone()
    pasta.convert(y, torch.float32, scale=sc, out=y)
    assert torch.equal(y, x * -1.75)
