"""Full-size workloads, in the launch configuration the benchmark times,
checked on sampled output rows that the oracle computes from the entries
that reach them (the generated tensor, never the GPU's sorted copy).

Sampled rows per mode: the heaviest row (the accuracy worst case), a few
random touched rows and, where one exists, an untouched row (must be 0).
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1902_03317_gb300 as pasta
from paper_1902_03317_gb300 import synth
from tests import _gpu as G

pytestmark = [pytest.mark.gpu, pytest.mark.fullsize]


def sample_rows(ix: np.ndarray, dim: int, rng, k: int = 6):
    counts = np.bincount(ix, minlength=dim)
    touched = np.flatnonzero(counts)
    rows = [int(np.argmax(counts))]
    rows += [int(r) for r in rng.choice(touched, size=min(k, touched.size), replace=False)]
    untouched = np.flatnonzero(counts == 0)
    if untouched.size:
        rows.append(int(untouched[rng.integers(0, untouched.size)]))
    return sorted(set(rows))


def subset(idx, val, mode, rows, dim):
    lut = np.zeros(dim, dtype=bool)
    lut[rows] = True
    keep = lut[idx[mode]]
    return [ix[keep] for ix in idx], val[keep]


def mttkrp_rows_check(name, dtypes, max_heavy=None):
    wl = synth.WORKLOADS[name]
    Xd = G.generate(wl, device=G.DEV)
    X = pasta.CooTensor(Xd.dims, Xd.idx, Xd.val)
    X.sort_all()
    idx = [i.cpu().numpy().astype(np.uint32) for i in Xd.idx]
    val = Xd.val.cpu().numpy().astype(np.float64)
    del Xd
    rng = np.random.default_rng(0)
    for dtype in dtypes:
        master = synth.factors_for(wl)
        dev = [u.to(dtype).to(G.DEV).contiguous() for u in master]
        rounded = [u.to(dtype).double().numpy() for u in master]
        for n in range(wl.order):
            M = pasta.mttkrp(X, dev, n)
            rows = sample_rows(idx[n], wl.dims[n], rng)
            if max_heavy is not None:
                rows = rows[:max_heavy] if wl.dims[n] <= max_heavy else rows
            sidx, sval = subset(idx, val, n, rows, wl.dims[n])
            ref = oracle.mttkrp(wl.dims, sidx, sval, rounded, n)[rows]
            got = M[torch.tensor(rows, device=G.DEV)].cpu().numpy()
            err = G.rel_err(got, ref)
            assert err < G.FP32_TOL, f"{name} {dtype} mode {n}: {err}"
            if dtype != torch.float32:
                ref_m = oracle.mttkrp(wl.dims, sidx, sval, [u.numpy() for u in master], n)[rows]
                assert G.rel_err(got, ref_m) < G.LOWP_TOL
    X.close()
    torch.cuda.empty_cache()


def test_zipf3d_100M_fp32():
    mttkrp_rows_check("zipf3d", [torch.float32, torch.bfloat16])


def test_zipf4d_50M_fp32_and_bf16():
    mttkrp_rows_check("zipf4d", [torch.float32, torch.bfloat16])


def test_zipf5d_200M_bf16():
    mttkrp_rows_check("zipf5d", [torch.bfloat16], max_heavy=3)


def test_cploss3d_20M_loss_and_grad():
    wl = synth.WORKLOADS["cploss3d"]
    Xd = G.generate(wl, device=G.DEV)
    X = pasta.CooTensor(Xd.dims, Xd.idx, Xd.val)
    X.sort_all()
    idx = [i.cpu().numpy().astype(np.uint32) for i in Xd.idx]
    val = Xd.val.cpu().numpy().astype(np.float64)
    del Xd
    rng = np.random.default_rng(1)
    for dtype in (torch.float32, torch.bfloat16):
        master = synth.factors_for(wl)
        dev = [u.to(dtype).to(G.DEV).contiguous() for u in master]
        rounded = [u.to(dtype).double().numpy() for u in master]
        loss = pasta.cp_loss_fwd(X, dev, 0).item()
        ref = oracle.cp_loss(wl.dims, idx, val, rounded)
        assert abs(loss - ref) <= G.FP32_TOL * ref
        for bwd_mode in (0, -2):
            grads = pasta.cp_loss_bwd(X, dev, bwd_mode)
            for k in range(3):
                rows = sample_rows(idx[k], wl.dims[k], rng)
                sidx, sval = subset(idx, val, k, rows, wl.dims[k])
                refg = oracle.cp_grad(wl.dims, sidx, sval, rounded)[k][rows]
                got = grads[k][torch.tensor(rows, device=G.DEV)].cpu().numpy()
                assert G.rel_err(got, refg) < G.FP32_TOL, (dtype, bwd_mode, k)
    X.close()
    torch.cuda.empty_cache()


def test_zipf3d_100M_als_sweep_normal_equations():
    """One CP-ALS sweep at full size.  After it, the last mode solves its
    least-squares problem: (U_2 diag(lam)) V = MTTKRP_2 with V the Hadamard
    product of the final U_0, U_1 Gram matrices, checked at sampled rows of
    MTTKRP_2 computed by the oracle from the entries reaching them.  Each
    column of every factor has unit norm, and since U_2 = 0 is a feasible
    update, 0 <= fit <= 1."""
    wl = synth.WORKLOADS["zipf3d"]
    Xd = G.generate(wl, device=G.DEV)
    X = pasta.CooTensor(Xd.dims, Xd.idx, Xd.val)
    idx = [i.cpu().numpy().astype(np.uint32) for i in Xd.idx]
    val = Xd.val.cpu().numpy().astype(np.float64)
    del Xd
    U = [u.to(G.DEV).contiguous() for u in synth.factors_for(wl)]
    lam, fit = pasta.cp_als_sweep(X, U)
    Uh = [u.cpu().double().numpy() for u in U]
    lam = lam.cpu().numpy()
    n = 2
    V = (Uh[0].T @ Uh[0]) * (Uh[1].T @ Uh[1])
    rows = sample_rows(idx[n], wl.dims[n], np.random.default_rng(1))
    sidx, sval = subset(idx, val, n, rows, wl.dims[n])
    M = oracle.mttkrp(wl.dims, sidx, sval, Uh, n)[rows]
    assert G.rel_err((Uh[n][rows] * lam[None, :]) @ V, M) < 1e-4
    for u in Uh:
        assert np.allclose(np.linalg.norm(u, axis=0), 1.0, atol=1e-5)
    assert 0.0 <= float(fit) <= 1.0
    X.close()
    torch.cuda.empty_cache()


def test_zipf3d_100M_tew_eq_and_ts_sampled():
    """TS and TEW-eq over the full 100M-entry tensor, checked at 1M sampled
    stored positions against the oracle (coordinates bit-exact, values within
    1 FP32 ulp; the multiplications exact)."""
    wl = synth.WORKLOADS["zipf3d"]
    Xd = G.generate(wl, device=G.DEV)
    X = pasta.CooTensor(Xd.dims, Xd.idx, Xd.val)
    del Xd
    Y = pasta.ts(X, "mul", -0.37)
    Z = pasta.tew_eq(X, Y, "div")
    rng = np.random.default_rng(3)
    pos = torch.tensor(np.sort(rng.choice(wl.nnz, size=1_000_000, replace=False)), device=G.DEV)
    xi, xv, _ = X.copy_out()
    _, yv, _ = Y.copy_out()
    zi, zv, _ = Z.copy_out()
    for k in range(3):
        assert torch.equal(zi[k], xi[k])
    idx_s = [xi[k][pos].cpu().numpy().astype(np.uint32) for k in range(3)]
    xs = xv[pos].cpu().double().numpy()
    _, ys = oracle.ts(idx_s, xs, "mul", float(np.float32(-0.37)))
    assert np.array_equal(yv[pos].cpu().numpy(), ys.astype(np.float32))
    _, zs = oracle.tew_eq(idx_s, xs, idx_s, yv[pos].cpu().double().numpy(), "div")
    from tests.test_gpu_tew import ulp_distance
    assert ulp_distance(zv[pos].cpu().numpy(), zs).max() <= 1
    for t in (X, Y, Z):
        t.close()
    torch.cuda.empty_cache()


def test_zipf3d_100M_ttm_sampled_fibers():
    """Mode-1 TTM (R = 32, FP32) of the full tensor: fiber count against the
    distinct (i_2, i_0) pairs, and sampled fibers (the heaviest and random
    ones) against the oracle run on the entries of those fibers."""
    wl = synth.WORKLOADS["zipf3d"]
    Xd = G.generate(wl, device=G.DEV)
    X = pasta.CooTensor(Xd.dims, Xd.idx, Xd.val)
    n = 1
    key = (Xd.idx[2].to(torch.int64) * wl.dims[0] + Xd.idx[0].to(torch.int64))
    uniq, counts = torch.unique(key, return_counts=True)
    idx = [i.cpu().numpy().astype(np.uint32) for i in Xd.idx]
    val = Xd.val.cpu().numpy().astype(np.float64)
    del Xd
    U = torch.randn(wl.dims[n], 32, device=G.DEV)
    Y = pasta.ttm(X, U, n)
    assert Y.shape[0] == uniq.numel()
    coords = pasta.fiber_coords(X, n)  # modes 2, 0
    fkey = coords[0].to(torch.int64) * wl.dims[0] + coords[1].to(torch.int64)
    assert torch.equal(fkey, uniq)  # sorted, distinct, complete
    rng = np.random.default_rng(4)
    pick = [int(torch.argmax(counts))] + [int(x) for x in rng.choice(uniq.numel(), 8, replace=False)]
    pkeys = fkey[pick].cpu().numpy()
    keys_h = key.cpu().numpy()
    keep = np.isin(keys_h, pkeys)
    sidx = [ix[keep] for ix in idx]
    c_ref, y_ref = oracle.ttm(wl.dims, sidx, val[keep], U.double().cpu().numpy(), n)
    ref_keys = c_ref[0].astype(np.int64) * wl.dims[0] + c_ref[1].astype(np.int64)
    order = np.argsort(pkeys)
    assert np.array_equal(ref_keys, pkeys[order])
    got = Y[torch.tensor(np.array(pick)[order], device=G.DEV)].cpu().numpy()
    assert G.rel_err(got, y_ref) < G.FP32_TOL
    X.close()
    torch.cuda.empty_cache()
