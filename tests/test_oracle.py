"""Pins for the FP64 oracle (CPU only).

The oracle is checked against things other than itself: a hand-worked example
(tests/golden), dense brute force through the Kolda matricization times the
Khatri-Rao product and through einsum, a closed form for rank-one tensors,
invariants, special cases and finite differences.  A battery of deliberately
broken MTTKRP/loss variants (planted mistakes, on the CPU) shows that each
plausible mistake fails at least one of these pins.
"""
from __future__ import annotations

import itertools

import numpy as np
import pytest

import oracle
from tests import _brute as brute

TIGHT = 1e-12


def rel_err(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


# ---------------------------------------------------------------- golden ---

def test_golden_worked_example_mttkrp(golden_worked):
    g = golden_worked
    for n in range(3):
        M = oracle.mttkrp(g["dims"], g["idx"], g["val"], g["U"], n, g["R"])
        np.testing.assert_array_equal(M, g[f"M{n}"])


def test_golden_worked_example_loss_and_grad(golden_worked):
    g = golden_worked
    loss, resid = oracle.cp_loss(g["dims"], g["idx"], g["val"], g["U"], want_resid=True)
    assert loss == g["loss"][0]
    np.testing.assert_array_equal(resid, g["resid"])
    G = oracle.cp_grad(g["dims"], g["idx"], g["val"], g["U"])
    for n in range(3):
        np.testing.assert_array_equal(G[n], g[f"G{n}"])


def test_golden_matches_matrix_form(golden_worked):
    """The hand-worked numbers agree with X_(n) (C o B) written with the
    explicit unfolding, so the fixture itself is consistent."""
    g = golden_worked
    X = brute.dense_from_coo(g["dims"], g["idx"], g["val"])
    for n in range(3):
        np.testing.assert_array_equal(brute.mttkrp_unfold(X, g["U"], n), g[f"M{n}"])


# ---------------------------------------------------------- brute force ---

CASES = []
for order in (3, 4, 5):
    for R in (1, 3, 4):
        CASES.append((order, R))


@pytest.mark.parametrize("order,R", CASES)
def test_mttkrp_vs_dense_brute_force(order, R):
    rng = np.random.default_rng(100 * order + R)
    dims = tuple(int(d) for d in rng.integers(2, 8 if order == 3 else (6 if order == 4 else 4), size=order))
    for density, dups in ((0.3, False), (1.0, False), (0.5, True)):
        idx, val = brute.random_coo(rng, dims, density, with_dups=dups)
        U = [rng.standard_normal((d, R)) for d in dims]
        X = brute.dense_from_coo(dims, idx, val)
        for n in range(order):
            M = oracle.mttkrp(dims, idx, val, U, n, R)
            assert rel_err(M, brute.mttkrp_unfold(X, U, n)) < TIGHT
            assert rel_err(M, brute.mttkrp_einsum(X, U, n)) < TIGHT


def test_rank_one_closed_form():
    """X = a^1 o a^2 o a^3 o a^4 with every cell stored:
    M_n(i, r) = a^n_i * prod_{k != n} <a^k, U_k(:, r)>."""
    rng = np.random.default_rng(7)
    dims = (3, 4, 2, 5)
    R = 3
    a = [rng.standard_normal(d) for d in dims]
    cells = np.array(list(itertools.product(*[range(d) for d in dims])))
    idx = [cells[:, k].astype(np.uint32) for k in range(4)]
    val = np.prod([a[k][cells[:, k]] for k in range(4)], axis=0)
    U = [rng.standard_normal((d, R)) for d in dims]
    for n in range(4):
        expect = np.outer(a[n], np.prod([a[k] @ U[k] for k in range(4) if k != n], axis=0))
        assert rel_err(oracle.mttkrp(dims, idx, val, U, n, R), expect) < TIGHT


def test_inner_product_invariant():
    """sum_{i,r} M_n(i,r) U_n(i,r) = sum_m x_m model_m, the same for every n."""
    rng = np.random.default_rng(11)
    dims = (9, 6, 7, 5)
    idx, val = brute.random_coo(rng, dims, 0.2, with_dups=True)
    R = 4
    U = [rng.standard_normal((d, R)) for d in dims]
    model = brute.cp_dense(U)[tuple(ix.astype(np.int64) for ix in idx)]
    target = float(np.sum(val * model))
    for n in range(4):
        got = float(np.sum(oracle.mttkrp(dims, idx, val, U, n, R) * U[n]))
        assert abs(got - target) <= 1e-11 * max(1.0, abs(target))


def test_all_ones_factors_give_slice_sums():
    rng = np.random.default_rng(12)
    dims = (8, 5, 6)
    idx, val = brute.random_coo(rng, dims, 0.4, with_dups=True)
    R = 3
    U = [np.ones((d, R)) for d in dims]
    for n in range(3):
        slice_sum = np.zeros(dims[n])
        np.add.at(slice_sum, idx[n].astype(np.int64), val)
        M = oracle.mttkrp(dims, idx, val, U, n, R)
        np.testing.assert_allclose(M, np.repeat(slice_sum[:, None], R, axis=1), rtol=0, atol=1e-13)


def test_columns_are_independent():
    rng = np.random.default_rng(13)
    dims = (7, 8, 9)
    idx, val = brute.random_coo(rng, dims, 0.3)
    R = 5
    U = [rng.standard_normal((d, R)) for d in dims]
    for n in range(3):
        M = oracle.mttkrp(dims, idx, val, U, n, R)
        for r in range(R):
            col = oracle.mttkrp(dims, idx, val, [u[:, r:r + 1] for u in U], n, 1)
            np.testing.assert_array_equal(M[:, r:r + 1], col)


def test_permutation_of_entries_and_duplicates():
    rng = np.random.default_rng(14)
    dims = (6, 7, 8)
    idx, val = brute.random_coo(rng, dims, 0.3)
    R = 4
    U = [rng.standard_normal((d, R)) for d in dims]
    p = rng.permutation(val.shape[0])
    # duplicate the first entry split into two halves: same result as one entry
    idx_d = [np.concatenate([ix, ix[:1]]) for ix in idx]
    val_d = np.concatenate([val, val[:1] * 0.5])
    val_d[0] *= 0.5
    for n in range(3):
        M = oracle.mttkrp(dims, idx, val, U, n, R)
        assert rel_err(oracle.mttkrp(dims, [ix[p] for ix in idx], val[p], U, n, R), M) < TIGHT
        assert rel_err(oracle.mttkrp(dims, idx_d, val_d, U, n, R), M) < TIGHT


def test_empty_tensor_gives_zero():
    dims = (3, 4, 5)
    idx = [np.zeros(0, dtype=np.uint32)] * 3
    U = [np.ones((d, 2)) for d in dims]
    for n in range(3):
        np.testing.assert_array_equal(oracle.mttkrp(dims, idx, np.zeros(0), U, n, 2), np.zeros((dims[n], 2)))
    assert oracle.cp_loss(dims, idx, np.zeros(0), U) == 0.0


# ------------------------------------------------------------ loss/grad ---

def test_loss_vs_dense_reconstruction():
    rng = np.random.default_rng(21)
    dims = (5, 6, 4, 3)
    idx, val = brute.random_coo(rng, dims, 0.4, with_dups=True)
    R = 3
    U = [rng.standard_normal((d, R)) for d in dims]
    model = brute.cp_dense(U)[tuple(ix.astype(np.int64) for ix in idx)]
    loss, resid = oracle.cp_loss(dims, idx, val, U, want_resid=True)
    np.testing.assert_allclose(resid, val - model, rtol=0, atol=1e-13)
    assert abs(loss - 0.5 * np.sum((val - model) ** 2)) < 1e-12 * max(1, loss)


def test_planted_exact_model_has_zero_loss_and_gradient():
    rng = np.random.default_rng(22)
    dims = (6, 5, 7)
    R = 3
    U = [rng.standard_normal((d, R)) for d in dims]
    cells = np.argwhere(rng.random(dims) < 0.5)
    idx = [cells[:, k].astype(np.uint32) for k in range(3)]
    val = brute.cp_dense(U)[tuple(cells.T)]
    assert oracle.cp_loss(dims, idx, val, U) < 1e-26
    for G in oracle.cp_grad(dims, idx, val, U):
        assert np.max(np.abs(G)) < 1e-12


def test_cp_model_values_match_dense_reconstruction():
    """The model evaluator behind the planted-value workload equals the dense
    CP tensor (Sec. 2.2) read at the coordinates, order 3 and 4."""
    rng = np.random.default_rng(24)
    for dims in ((6, 5, 7), (4, 3, 5, 2)):
        U = [rng.standard_normal((d, 3)) for d in dims]
        cells = np.argwhere(rng.random(dims) < 0.6)
        idx = [cells[:, k].astype(np.uint32) for k in range(len(dims))]
        got = oracle.cp_model_values(dims, idx, U)
        assert np.max(np.abs(got - brute.cp_dense(U)[tuple(cells.T)])) < 1e-12


def test_gradient_is_minus_mttkrp_of_residual():
    rng = np.random.default_rng(23)
    dims = (5, 4, 6)
    idx, val = brute.random_coo(rng, dims, 0.5)
    R = 2
    U = [rng.standard_normal((d, R)) for d in dims]
    _, resid = oracle.cp_loss(dims, idx, val, U, want_resid=True)
    G = oracle.cp_grad(dims, idx, val, U, g=2.5)
    X_e = brute.dense_from_coo(dims, idx, resid)
    for n in range(3):
        assert rel_err(G[n], -2.5 * brute.mttkrp_einsum(X_e, U, n)) < TIGHT


@pytest.mark.parametrize("order", [3, 4])
def test_gradient_finite_differences(order):
    """Central differences of the FP64 loss, h = 1e-6, on every factor entry."""
    rng = np.random.default_rng(30 + order)
    dims = (4, 3, 5, 3)[:order]
    idx, val = brute.random_coo(rng, dims, 0.5, with_dups=True)
    R = 3
    U = [rng.standard_normal((d, R)) for d in dims]
    G = oracle.cp_grad(dims, idx, val, U)
    h = 1e-6
    for n in range(order):
        fd = np.zeros_like(U[n])
        for i in range(dims[n]):
            for r in range(R):
                Up = [u.copy() for u in U]
                Um = [u.copy() for u in U]
                Up[n][i, r] += h
                Um[n][i, r] -= h
                fd[i, r] = (oracle.cp_loss(dims, idx, val, Up) - oracle.cp_loss(dims, idx, val, Um)) / (2 * h)
        assert rel_err(G[n], fd) < 1e-7


# ----------------------------------------------------------------- sort ---

def test_sort_perm_matches_python_sorted():
    rng = np.random.default_rng(40)
    dims = (4, 3, 5, 2)
    idx, _ = brute.random_coo(rng, dims, 0.6, with_dups=True)
    nnz = idx[0].shape[0]
    for mode in range(4):
        order = oracle.mode_order(4, mode)
        expect = sorted(range(nnz), key=lambda m: (tuple(int(idx[k][m]) for k in order), m))
        np.testing.assert_array_equal(oracle.sort_perm(idx, mode), np.array(expect))


# ------------------------------------------------- planted mistakes -------

def _mttkrp_loop(dims, idx, val, U, n, R, mistake=None):
    """Element-wise MTTKRP in pure Python with an optional planted mistake."""
    M = np.zeros((dims[n], R))
    N = len(dims)
    others = [k for k in range(N) if k != n]
    for m in range(val.shape[0]):
        for r in range(R):
            t = val[m]
            for j, k in enumerate(others):
                if mistake == "dropped_factor" and j == 0:
                    continue
                i_k = (int(idx[n][m]) % dims[k]) if (mistake == "wrong_index" and j == 0) else int(idx[k][m])
                if mistake == "transposed":
                    flat = U[k].T.reshape(-1)
                    t *= flat[(i_k * R + r) % flat.shape[0]]
                else:
                    t *= U[k][i_k, r]
            row = int(idx[n][m])
            if mistake == "off_by_one_row":
                row = (row + 1) % dims[n]
            if mistake == "sign":
                M[row, r] -= t
            else:
                M[row, r] += t
    return M


def _mttkrp_pins_pass(fn, golden) -> bool:
    """Run the MTTKRP pins against ``fn``; True only if every pin holds."""
    g = golden
    for n in range(3):
        if not np.array_equal(fn(g["dims"], g["idx"], g["val"], g["U"], n, g["R"]), g[f"M{n}"]):
            return False
    rng = np.random.default_rng(5)
    dims = (4, 5, 3)
    idx, val = brute.random_coo(rng, dims, 0.5)
    U = [rng.standard_normal((d, 3)) for d in dims]
    X = brute.dense_from_coo(dims, idx, val)
    for n in range(3):
        if rel_err(fn(dims, idx, val, U, n, 3), brute.mttkrp_einsum(X, U, n)) > 1e-10:
            return False
    return True


@pytest.mark.parametrize("mistake", ["dropped_factor", "wrong_index", "transposed", "off_by_one_row", "sign"])
def test_pins_catch_planted_mttkrp_mistakes(golden_worked, mistake):
    assert _mttkrp_pins_pass(lambda *a: _mttkrp_loop(*a), golden_worked)
    assert _mttkrp_pins_pass(lambda *a: oracle.mttkrp(*a), golden_worked)
    assert not _mttkrp_pins_pass(lambda *a: _mttkrp_loop(*a, mistake=mistake), golden_worked)


def _loss_grad_loop(dims, idx, val, U, mistake=None):
    N = len(dims)
    R = U[0].shape[1]
    loss = 0.0
    G = [np.zeros_like(u) for u in U]
    for m in range(val.shape[0]):
        rows = [U[k][int(idx[k][m])] for k in range(N)]
        model = float(np.sum(np.prod(rows, axis=0)))
        if mistake == "model_drops_last_mode":
            model = float(np.sum(np.prod(rows[:-1], axis=0)))
        e = val[m] - model
        loss += (e * e) if mistake == "no_half" else 0.5 * e * e
        for n in range(N):
            p = np.prod([rows[k] for k in range(N) if k != n], axis=0)
            G[n][int(idx[n][m])] += (e if mistake == "grad_sign" else -e) * p
    return loss, G


@pytest.mark.parametrize("mistake", ["no_half", "grad_sign", "model_drops_last_mode"])
def test_pins_catch_planted_loss_mistakes(golden_worked, mistake):
    g = golden_worked

    def passes(fn):
        loss, G = fn(g["dims"], g["idx"], g["val"], g["U"])
        return loss == g["loss"][0] and all(np.array_equal(G[n], g[f"G{n}"]) for n in range(3))

    assert passes(_loss_grad_loop)
    assert passes(lambda *a: (oracle.cp_loss(*a), oracle.cp_grad(*a)))
    assert not passes(lambda *a: _loss_grad_loop(*a, mistake=mistake))


# ---------------------------------------------------------------------------
# The multicore CPU baseline (privatization MTTKRP of Sec. 5.3, FP32) is a
# timed baseline, not a reference; it must still compute the same MTTKRP.

@pytest.mark.parametrize("threads", [1, 3, 0])
def test_cpu_privatized_baseline_matches_oracle(threads):
    rng = np.random.default_rng(5)
    dims = (40, 30, 20, 6)
    nnz = 3000
    idx = [rng.integers(0, d, nnz).astype(np.uint32) for d in dims]
    val = rng.standard_normal(nnz)
    U = [rng.standard_normal((d, 8)) for d in dims]
    Uf = [u.astype(np.float32) for u in U]
    for n in range(len(dims)):
        ref = oracle.mttkrp(dims, idx, val.astype(np.float32).astype(np.float64),
                            [u.astype(np.float64) for u in Uf], n, 8)
        got = oracle.mttkrp_privatized(dims, idx, val, Uf, n, threads=threads)
        assert got.dtype == np.float32
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-5
