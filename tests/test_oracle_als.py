"""Pins for the oracle's CP-ALS sweep (CPU only).

The sweep is checked against properties fixed by the mathematics rather than
by its own formulas: the least-squares optimality (normal equations) of each
mode update, unit columns, the closed form for rank-one tensors, the fit
against a dense reconstruction, exact recovery of a planted CP model, and the
monotone fit of alternating least squares.  Deliberately broken sweeps
(planted mistakes, on the CPU) show that each plausible mistake fails one of
these pins.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from tests import _brute as brute


def rel_err(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def _dense_model(dims, U, lam):
    letters = "abcdefgh"[: len(dims)]
    spec = ",".join(f"{c}r" for c in letters) + ",r->" + letters
    return np.einsum(spec, *U, lam)


def _fully_stored(X):
    idx = [ix.ravel().astype(np.uint32) for ix in np.indices(X.shape)]
    return idx, X.ravel().astype(np.float64)


# ----------------------------------------------------- the sweep under test --

def _sweep_py(dims, idx, val, U, mistake=None):
    """CP-ALS sweep restated in plain numpy with an optional planted mistake;
    without one it must agree with ``oracle.cp_als_sweep``."""
    N = len(dims)
    U = [np.array(u, dtype=np.float64, copy=True) for u in U]
    U_old = [u.copy() for u in U]
    R = U[0].shape[1]
    lam = np.ones(R)
    M = None
    for n in range(N):
        src = U_old if mistake == "stale_factors" else U
        M = oracle.mttkrp(dims, idx, val, src, n, R)
        V = np.ones((R, R))
        for j, k in enumerate([k for k in range(N) if k != n]):
            if mistake == "dropped_gram" and j == 0:
                continue
            V *= src[k].T @ src[k]
        Un = M @ V if mistake == "multiply_not_solve" else np.linalg.solve(V, M.T).T
        lam = np.linalg.norm(Un, axis=0)
        U[n] = Un if mistake == "no_normalize" else Un / np.where(lam > 0, lam, 1.0)
    normx2 = float(val @ val)
    H = np.ones((R, R))
    for u in U:
        H *= u.T @ u
    inner = float(np.sum(lam * np.sum(M * U[-1], axis=0)))
    two = 1.0 if mistake == "fit_inner_once" else 2.0
    fit = 1.0 - np.sqrt(max(normx2 + lam @ H @ lam - two * inner, 0.0)) / np.sqrt(normx2)
    return U, lam, fit


# ------------------------------------------------------------------- pins ---

def _pin_normal_equations(sweep) -> bool:
    """After the sweep the last mode solves its least-squares problem:
    (U_{N-1} diag(lam)) V = MTTKRP_{N-1} with the final other factors."""
    rng = np.random.default_rng(11)
    dims = (7, 6, 5)
    idx, val = brute.random_coo(rng, dims, 0.4)
    U0 = [rng.standard_normal((d, 3)) for d in dims]
    U, lam, _ = sweep(dims, idx, val, U0)
    n = 2
    M = oracle.mttkrp(dims, idx, val, U, n, 3)
    V = (U[0].T @ U[0]) * (U[1].T @ U[1])
    return rel_err((U[n] * lam[None, :]) @ V, M) < 1e-10


def _pin_unit_columns(sweep) -> bool:
    rng = np.random.default_rng(12)
    dims = (6, 5, 4, 3)
    idx, val = brute.random_coo(rng, dims, 0.5)
    U, _, _ = sweep(dims, idx, val, [rng.standard_normal((d, 2)) for d in dims])
    return all(np.allclose(np.linalg.norm(u, axis=0), 1.0, atol=1e-12) for u in U)


def _pin_rank_one_closed_form(sweep) -> bool:
    """For X = a o b o c fully stored, the first update of every mode is
    already proportional to the planted vector, so one sweep gives fit 1 and
    lam = ||a|| ||b|| ||c||."""
    rng = np.random.default_rng(13)
    a, b, c = (rng.uniform(0.5, 2.0, d) for d in (5, 4, 3))
    X = np.einsum("i,j,k->ijk", a, b, c)
    idx, val = _fully_stored(X)
    U0 = [rng.uniform(0.1, 1.0, (d, 1)) for d in X.shape]
    U, lam, fit = sweep(X.shape, idx, val, U0)
    ok = abs(fit - 1.0) < 1e-12 and abs(lam[0] - np.prod([np.linalg.norm(v) for v in (a, b, c)])) < 1e-10 * lam[0]
    for u, v in zip(U, (a, b, c)):
        ok = ok and rel_err(u[:, 0], v / np.linalg.norm(v)) < 1e-12
    return ok


def _pin_fit_vs_dense(sweep) -> bool:
    """The fit equals 1 - ||X - model||_F / ||X||_F from a dense
    reconstruction (zeros included) of a tensor with distinct coordinates."""
    rng = np.random.default_rng(14)
    dims = (5, 4, 6)
    idx, val = brute.random_coo(rng, dims, 0.5)
    X = brute.dense_from_coo(dims, idx, val)
    U, lam, fit = sweep(dims, idx, val, [rng.standard_normal((d, 3)) for d in dims])
    fit_bf = 1.0 - np.linalg.norm(X - _dense_model(dims, U, lam)) / np.linalg.norm(X)
    return abs(fit - fit_bf) < 1e-12


def _pin_monotone(sweep) -> bool:
    """Each mode update minimises the objective over that factor exactly, so
    the fit never decreases from sweep to sweep."""
    rng = np.random.default_rng(15)
    dims = (6, 7, 5)
    idx, val = brute.random_coo(rng, dims, 0.5)
    U = [rng.standard_normal((d, 3)) for d in dims]
    fits = []
    for _ in range(6):
        U, _, fit = sweep(dims, idx, val, U)
        fits.append(fit)
    return all(f1 >= f0 - 1e-12 for f0, f1 in zip(fits, fits[1:]))


PINS = [_pin_normal_equations, _pin_unit_columns, _pin_rank_one_closed_form, _pin_fit_vs_dense,
        _pin_monotone]


@pytest.mark.parametrize("pin", PINS, ids=lambda p: p.__name__[5:])
def test_oracle_sweep_holds_pin(pin):
    assert pin(oracle.cp_als_sweep)


def test_restated_sweep_matches_oracle():
    rng = np.random.default_rng(16)
    dims = (6, 5, 7)
    idx, val = brute.random_coo(rng, dims, 0.5)
    U0 = [rng.standard_normal((d, 4)) for d in dims]
    Ua, la, fa = oracle.cp_als_sweep(dims, idx, val, U0)
    Ub, lb, fb = _sweep_py(dims, idx, val, U0)
    assert all(rel_err(a, b) < 1e-12 for a, b in zip(Ua, Ub))
    assert rel_err(la, lb) < 1e-12 and abs(fa - fb) < 1e-12


def test_planted_model_is_recovered():
    rng = np.random.default_rng(17)
    A = [rng.standard_normal((d, 2)) for d in (6, 5, 4)]
    X = np.einsum("ir,jr,kr->ijk", *A)
    idx, val = _fully_stored(X)
    U = [a + 1e-3 * rng.standard_normal(a.shape) for a in A]
    fit = 0.0
    for _ in range(60):
        U, lam, fit = oracle.cp_als_sweep(X.shape, idx, val, U)
    assert fit > 1.0 - 1e-7
    assert rel_err(_dense_model(X.shape, U, lam), X) < 1e-7


def test_zero_column_makes_the_next_solve_singular():
    """A factor column the stored entries never reach comes out of its update
    as zeros (lam = 0, no division by zero); the next mode's V then has a zero
    row and column, and the inverse does not exist: the sweep reports it."""
    dims = (3, 3, 3)
    idx = [np.array([0, 1], dtype=np.uint32)] * 3
    val = np.array([1.0, 2.0])
    U0 = [np.eye(3)[:, :2] for _ in dims]
    U0[1] = np.array([[1.0, 0.0], [0.0, 0.0], [0.0, 1.0]])  # column 1 only at row 2, never stored
    U0[2] = U0[1].copy()
    with pytest.raises(np.linalg.LinAlgError):
        oracle.cp_als_sweep(dims, idx, val, U0)


@pytest.mark.parametrize("mistake", ["stale_factors", "dropped_gram", "multiply_not_solve",
                                     "no_normalize", "fit_inner_once"])
def test_pins_catch_planted_als_mistakes(mistake):
    assert all(pin(_sweep_py) for pin in PINS)
    broken = lambda *a: _sweep_py(*a, mistake=mistake)  # noqa: E731
    assert not all(pin(broken) for pin in PINS)
