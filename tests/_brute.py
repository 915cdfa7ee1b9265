"""Dense brute-force restatements used to pin the oracle (tiny tensors only).

These follow the matrix form of the definitions rather than the element-wise
loop of the oracle:
  - mode-n matricization in the Kolda-Bader convention (X_(n) is
    I_n x prod_{k!=n} I_k, the first remaining mode varying fastest); the
    paper's Sec. 3 prints the transposed shape, which cannot multiply the
    Khatri-Rao product in Eq. (mttkrp-init), so the Kolda reading is taken;
  - the Khatri-Rao product as the column-wise Kronecker product (Sec. 3.5),
    in the order U_N o ... o U_{n+1} o U_{n-1} o ... o U_1 of Eq. (mttkrp-init);
  - np.einsum over the dense tensor as a second, independent route.
"""
from __future__ import annotations

import string

import numpy as np


def dense_from_coo(dims, idx, val) -> np.ndarray:
    X = np.zeros(tuple(int(d) for d in dims), dtype=np.float64)
    np.add.at(X, tuple(np.asarray(ix, dtype=np.int64) for ix in idx), np.asarray(val, dtype=np.float64))
    return X


def unfold(X: np.ndarray, n: int) -> np.ndarray:
    """Kolda-Bader mode-n matricization: rows = mode n, columns ordered with
    the lowest remaining mode varying fastest."""
    return np.reshape(np.moveaxis(X, n, 0), (X.shape[n], -1), order="F")


def khatri_rao(mats) -> np.ndarray:
    """Column-wise Kronecker product of the matrices in the given order
    (the first matrix varies slowest)."""
    R = mats[0].shape[1]
    cols = []
    for r in range(R):
        c = np.ones(1)
        for A in mats:
            c = np.kron(c, A[:, r])
        cols.append(c)
    return np.stack(cols, axis=1)


def mttkrp_unfold(X: np.ndarray, U, n: int) -> np.ndarray:
    N = X.ndim
    mats = [U[k] for k in reversed(range(N)) if k != n]
    return unfold(X, n) @ khatri_rao(mats)


def mttkrp_einsum(X: np.ndarray, U, n: int) -> np.ndarray:
    N = X.ndim
    letters = string.ascii_lowercase[:N]
    terms = [letters] + [letters[k] + "z" for k in range(N) if k != n]
    spec = ",".join(terms) + "->" + letters[n] + "z"
    return np.einsum(spec, X, *[U[k] for k in range(N) if k != n])


def cp_dense(U) -> np.ndarray:
    """Dense rank-R CP reconstruction sum_r a^1_r o ... o a^N_r via einsum."""
    N = len(U)
    letters = string.ascii_lowercase[:N]
    spec = ",".join(l + "z" for l in letters) + "->" + letters
    return np.einsum(spec, *U)


def random_coo(rng: np.random.Generator, dims, density: float, with_dups: bool = False):
    """Random COO over a small dense grid: each cell stored with probability
    ``density``; optional duplicated entries appended."""
    cells = np.argwhere(rng.random(dims) < density)
    if cells.shape[0] == 0:
        cells = np.zeros((1, len(dims)), dtype=np.int64)
    if with_dups:
        extra = cells[rng.integers(0, cells.shape[0], size=max(1, cells.shape[0] // 3))]
        cells = np.concatenate([cells, extra])
    rng.shuffle(cells)
    idx = [cells[:, k].astype(np.uint32) for k in range(len(dims))]
    val = rng.uniform(-1, 1, size=cells.shape[0])
    return idx, val
