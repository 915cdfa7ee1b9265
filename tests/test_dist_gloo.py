"""Multi-rank partition logic on CPU (gloo, world size 2), checked with the oracle.

Row-aligned ranges of the mode-sorted stream give each rank a disjoint block of
output rows (no reduction); arbitrary ranges need a sum all-reduce of the
partial outputs (the paper's privatization, Sec. 5.3), as does the data-parallel
loss gradient.  No GPU is involved.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_1902_03317_gb300 import shard, synth


def _tensor():
    wl = synth.WORKLOADS["zipf3d"].scaled(nnz=4000, dims=(300, 200, 100))
    X = synth.generate(wl)
    idx = [i.numpy().astype(np.uint32) for i in X.idx]
    val = X.val.numpy().astype(np.float64)
    U = [u.double().numpy() for u in synth.factors_for(wl, R=4)]
    return wl.dims, idx, val, U


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, results):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dims, idx, val, U = _tensor()
        mode = 0
        p = oracle.sort_perm(idx, mode)
        sidx = [ix[p] for ix in idx]
        sval = val[p]
        # row-aligned: disjoint output rows, then a sum is the same as a gather
        lo, hi = shard.row_aligned_ranges(sidx[mode], world)[rank]
        M = oracle.mttkrp(dims, [ix[lo:hi] for ix in sidx], sval[lo:hi], U, mode)
        owned = np.flatnonzero(np.abs(M).sum(axis=1))
        t = torch.from_numpy(M)
        dist.all_reduce(t)
        rows_t = torch.zeros(dims[mode], dtype=torch.int64)
        rows_t[torch.from_numpy(owned)] = 1
        dist.all_reduce(rows_t)
        # arbitrary ranges + all-reduce (privatization)
        lo2, hi2 = shard.even_ranges(len(val), world)[rank]
        M2 = torch.from_numpy(oracle.mttkrp(dims, [ix[lo2:hi2] for ix in idx], val[lo2:hi2], U, mode))
        dist.all_reduce(M2)
        # data-parallel loss gradient
        G = [torch.from_numpy(g) for g in oracle.cp_grad(dims, [ix[lo2:hi2] for ix in idx], val[lo2:hi2], U)]
        loss = torch.tensor([oracle.cp_loss(dims, [ix[lo2:hi2] for ix in idx], val[lo2:hi2], U)], dtype=torch.float64)
        for g in G:
            dist.all_reduce(g)
        dist.all_reduce(loss)
        if rank == 0:
            results.put((t.numpy(), int(rows_t.max()), M2.numpy(), [g.numpy() for g in G], float(loss[0])))
    finally:
        dist.destroy_process_group()


def test_row_aligned_ranges_never_split_rows():
    rng = np.random.default_rng(0)
    rows = np.sort(rng.integers(0, 50, size=1000))
    for parts in (1, 2, 3, 7, 64):
        rs = shard.row_aligned_ranges(rows, parts)
        assert rs[0][0] == 0 and rs[-1][1] == 1000
        for (a, b), (c, d) in zip(rs, rs[1:]):
            assert b == c and a <= b
            if 0 < b < 1000:
                assert rows[b - 1] != rows[b]
    # one row holding everything: all entries in one range
    rs = shard.row_aligned_ranges(np.zeros(100, dtype=int), 4)
    assert sorted(b - a for a, b in rs) == [0, 0, 0, 100]
    with pytest.raises(ValueError):
        shard.row_aligned_ranges(np.array([3, 1]), 2)


def test_even_ranges_cover():
    rs = shard.even_ranges(10, 3)
    assert rs == [(0, 3), (3, 6), (6, 10)]


def test_two_gloo_ranks_match_whole_tensor():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    M_sum, max_owner, M_priv, G, loss = q.get(timeout=120)
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    dims, idx, val, U = _tensor()
    ref = oracle.mttkrp(dims, idx, val, U, 0)
    np.testing.assert_allclose(M_sum, ref, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(M_priv, ref, rtol=1e-12, atol=1e-12)
    assert max_owner == 1  # every output row owned by at most one rank
    for g, r in zip(G, oracle.cp_grad(dims, idx, val, U)):
        np.testing.assert_allclose(g, r, rtol=1e-12, atol=1e-12)
    assert abs(loss - oracle.cp_loss(dims, idx, val, U)) < 1e-9 * max(1.0, loss)


def _worker_step(rank, world, port, results):
    """The sharded step of bench.py on gloo ranks with oracle arithmetic:
    each rank takes shard.step_range of every mode's sorted copy, computes
    its partial MTTKRP for every mode and its partial loss and gradients, and
    completes the range-end rows with shard.complete_boundary_rows."""
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dims, idx, val, U = _tensor()
        nnz = len(val)
        lo, hi = shard.step_range(nnz, world, rank)
        Ms, Gs, loss = [], [], 0.0
        for n in range(len(dims)):
            p = oracle.sort_perm(idx, n)
            sidx = [ix[p][lo:hi] for ix in idx]
            sval = val[p][lo:hi]
            M = torch.from_numpy(oracle.mttkrp(dims, sidx, sval, U, n))
            first = int(sidx[n][0]) if hi > lo else -1
            last = int(sidx[n][-1]) if hi > lo else -1
            shard.complete_boundary_rows(M, first, last)
            G = torch.from_numpy(oracle.cp_grad(dims, sidx, sval, U)[n])
            shard.complete_boundary_rows(G, first, last)
            reach = np.unique(sidx[n])
            Ms.append((M.numpy()[reach], reach))
            Gs.append((G.numpy()[reach], reach))
            if n == 0:
                loss = oracle.cp_loss(dims, sidx, sval, U)
        lt = torch.tensor([loss], dtype=torch.float64)
        dist.all_reduce(lt)
        results.put((rank, Ms, Gs, float(lt[0])))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_step_matches_whole_tensor(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker_step, args=(r, world, port, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    got = [q.get(timeout=180) for _ in range(world)]
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    dims, idx, val, U = _tensor()
    refG = oracle.cp_grad(dims, idx, val, U)
    for rank, Ms, Gs, loss in got:
        assert abs(loss - oracle.cp_loss(dims, idx, val, U)) < 1e-9 * max(1.0, loss)
        for n in range(len(dims)):
            ref = oracle.mttkrp(dims, idx, val, U, n)
            m, rows = Ms[n]
            np.testing.assert_allclose(m, ref[rows], rtol=1e-12, atol=1e-12)
            g, rows = Gs[n]
            np.testing.assert_allclose(g, refG[n][rows], rtol=1e-12, atol=1e-12)
    # together the ranks reach every row that has an entry
    for n in range(len(dims)):
        reached = set()
        for _, Ms, _, _ in got:
            reached |= set(Ms[n][1].tolist())
        assert reached == set(np.unique(idx[n]).tolist())


def test_aligned_ranges_cover():
    for nnz in (0, 1, 3, 4, 10, 4001, 100_003):
        for parts in (1, 2, 3, 8):
            rs = shard.aligned_ranges(nnz, parts)
            assert rs[0][0] == 0 and rs[-1][1] == nnz and len(rs) == parts
            for (a, b), (c, d) in zip(rs, rs[1:]):
                assert b == c and a <= b and a % 4 == 0
            assert max(b - a for a, b in rs) - min(b - a for a, b in rs) <= 4 * 2 or nnz < 8 * parts
