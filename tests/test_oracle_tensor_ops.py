"""Pins for the oracle's TEW-eq, TS, TTV and TTM (CPU only).

TEW-eq and TS (Algorithms 1 and 3) are checked against dense element-wise
arithmetic on the support and against algebraic identities; TTV and TTM
(Algorithms 4 and 5) against dense einsum contractions, the matricized form
Y_(n) = U^T X_(n) of Eq. (moden-mat) written with the unfolding, the set of
distinct fibers, and each other.  Deliberately broken versions (planted
mistakes, on the CPU) must fail at least one pin.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from tests import _brute as brute


def _distinct(rng, dims, density):
    idx, val = brute.random_coo(rng, dims, density)
    keys = np.stack(idx, axis=1)
    _, first = np.unique(keys, axis=0, return_index=True)
    first = np.sort(first)
    return [ix[first] for ix in idx], val[first]


# ------------------------------------------------------------ TEW-eq / TS ---

def _tew_py(idx_x, vx, idx_y, vy, op, mistake=None):
    vx = np.asarray(vx, dtype=np.float64)
    vy = np.asarray(vy, dtype=np.float64)
    if mistake == "swapped_sub" and op == "sub":
        return vy - vx
    if mistake == "inverted_div" and op == "div":
        return vy / vx
    if mistake == "mul_is_add" and op == "mul":
        return vx + vy
    return oracle.tew_eq(idx_x, vx, idx_y, vy, op)[1]


def _ts_py(idx_x, vx, op, s, mistake=None):
    vx = np.asarray(vx, dtype=np.float64)
    if mistake == "ts_add_scales" and op == "add":
        return vx * s
    if mistake == "ts_div_multiplies" and op == "div":
        return vx * s
    return oracle.ts(idx_x, vx, op, s)[1]


def _tew_pins(tew, ts) -> bool:
    rng = np.random.default_rng(31)
    dims = (5, 4, 6)
    idx, vx = _distinct(rng, dims, 0.5)
    vy = rng.uniform(0.5, 2.0, vx.shape) * rng.choice([-1.0, 1.0], vx.shape)
    X = brute.dense_from_coo(dims, idx, vx)
    Y = brute.dense_from_coo(dims, idx, vy)
    sup = tuple(np.asarray(ix, dtype=np.int64) for ix in idx)
    with np.errstate(divide="ignore", invalid="ignore"):
        dense = {"add": X + Y, "sub": X - Y, "mul": X * Y, "div": X / Y}
    for op in oracle.OPS:
        if not np.allclose(tew(idx, vx, idx, vy, op), dense[op][sup], rtol=1e-14, atol=0):
            return False
    s = -1.75
    with np.errstate(divide="ignore"):
        dense_s = {"add": X + s, "sub": X - s, "mul": X * s, "div": X / s}
    for op in oracle.OPS:
        if not np.allclose(ts(idx, vx, op, s), dense_s[op][sup], rtol=1e-14, atol=0):
            return False
    # identities on the stored values
    if not np.allclose(tew(idx, tew(idx, vx, idx, vy, "add"), idx, vy, "sub"), vx, rtol=1e-14, atol=1e-15):
        return False
    if not np.array_equal(ts(idx, ts(idx, vx, "add", 3.0), "sub", 3.0), vx + 3.0 - 3.0):
        return False
    return np.allclose(ts(idx, vx, "div", 4.0), ts(idx, vx, "mul", 0.25), rtol=1e-15, atol=0)


def test_tew_ts_oracle_pins():
    assert _tew_pins(_tew_py, _ts_py)


def test_tew_eq_rejects_different_coordinates():
    rng = np.random.default_rng(32)
    idx, v = _distinct(rng, (4, 4, 4), 0.5)
    idx2 = [ix.copy() for ix in idx]
    idx2[1][0] = (idx2[1][0] + 1) % 4
    with pytest.raises(ValueError):
        oracle.tew_eq(idx, v, idx2, v, "add")


@pytest.mark.parametrize("mistake", ["swapped_sub", "inverted_div", "mul_is_add", "ts_add_scales",
                                     "ts_div_multiplies"])
def test_tew_ts_pins_catch_planted_mistakes(mistake):
    broken_tew = lambda *a: _tew_py(*a, mistake=mistake)  # noqa: E731
    broken_ts = lambda *a: _ts_py(*a, mistake=mistake)    # noqa: E731
    assert not _tew_pins(broken_tew, broken_ts)


# -------------------------------------------------------------- TTV / TTM ---

def _ttm_py(dims, idx, val, U, mode, mistake=None):
    """Mode-n TTM restated with a dictionary, with an optional mistake."""
    N = len(dims)
    U = np.asarray(U, dtype=np.float64)
    modes = oracle.fiber_modes(N, mode)
    acc = {}
    for m in range(len(val)):
        key = tuple(int(idx[k][m]) for k in modes)
        if mistake == "fiber_includes_n":
            key = key + (int(idx[mode][m]),)
        i_n = int(idx[mode][m])
        if mistake == "wrong_row_mode":
            i_n = int(idx[modes[0]][m]) % U.shape[0]
        x = 1.0 if mistake == "dropped_value" else float(val[m])
        row = U[:, 0] if mistake == "transposed" else U[i_n]
        acc[key] = acc.get(key, 0.0) + x * (row[: U.shape[1]] if mistake == "transposed" else row)
    keys = sorted(acc)
    if mistake == "fiber_includes_n":
        keys = sorted(acc)
        Y = np.array([acc[k] for k in keys])
        return [np.array([k[j] for k in keys], dtype=np.uint32) for j in range(N)], Y
    Y = np.array([acc[k] for k in keys]) if keys else np.zeros((0, U.shape[1]))
    return [np.array([k[j] for k in keys], dtype=np.uint32) for j in range(N - 1)], Y


def _ttm_pins(ttm) -> bool:
    rng = np.random.default_rng(41)
    for dims in ((4, 5, 3), (3, 4, 2, 5)):
        N = len(dims)
        idx, val = brute.random_coo(rng, dims, 0.45, with_dups=True)  # duplicates add
        X = brute.dense_from_coo(dims, idx, val)
        for mode in range(N):
            R = 3
            U = rng.standard_normal((dims[mode], R))
            coords, Y = ttm(dims, idx, val, U, mode)
            modes = oracle.fiber_modes(N, mode)
            # the fibers are exactly the distinct coordinates without i_n, in
            # lexicographic order of the cyclic modes
            distinct = sorted({tuple(int(idx[k][m]) for k in modes) for m in range(len(val))})
            got = list(zip(*[c.tolist() for c in coords])) if len(coords) == N - 1 else None
            if got != distinct:
                return False
            # dense contraction along mode n (Eq. (ttm)), read at the fibers
            Yd = np.moveaxis(np.tensordot(X, U, axes=([mode], [0])), -1, 0)  # R x (dims without n)
            rest = [k for k in range(N) if k != mode]
            pos = [rest.index(k) for k in modes]
            want = np.stack([Yd[(slice(None),) + tuple(np.array(f)[np.argsort(pos)])] for f in distinct])
            if not np.allclose(Y, want, rtol=1e-12, atol=1e-12):
                return False
            # matricized form: Y_(n) = U^T X_(n) (Kolda unfolding)
            Xn = brute.unfold(X, mode)
            Yn = U.T @ Xn
            cols = [int(sum(f[rest.index(k)] * int(np.prod([dims[j] for j in rest[: rest.index(k)]]))
                            for k in rest)) for f in [tuple(np.array(fd)[np.argsort(pos)]) for fd in distinct]]
            if not np.allclose(Y, Yn[:, cols].T, rtol=1e-12, atol=1e-12):
                return False
    return True


def test_ttm_oracle_pins():
    assert _ttm_pins(oracle.ttm)
    assert _ttm_pins(_ttm_py)


def test_ttv_is_ttm_with_one_column():
    rng = np.random.default_rng(42)
    dims = (6, 5, 4)
    idx, val = brute.random_coo(rng, dims, 0.4)
    v = rng.standard_normal(dims[2])
    c1, y = oracle.ttv(dims, idx, val, v, 2)
    c2, Y = oracle.ttm(dims, idx, val, v[:, None], 2)
    assert all(np.array_equal(a, b) for a, b in zip(c1, c2)) and np.array_equal(y, Y[:, 0])
    # TTV against the dense contraction, read at the fibers
    X = brute.dense_from_coo(dims, idx, val)
    Yd = np.tensordot(X, v, axes=([2], [0]))
    assert np.allclose(y, Yd[c1[0].astype(int), c1[1].astype(int)], rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("mistake", ["fiber_includes_n", "wrong_row_mode", "dropped_value", "transposed"])
def test_ttm_pins_catch_planted_mistakes(mistake):
    assert not _ttm_pins(lambda *a: _ttm_py(*a, mistake=mistake))
