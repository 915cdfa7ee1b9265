"""FP64 CPU oracle for COO MTTKRP, the sparse CP loss and its gradient.

TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT.  Only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` may import this package.  It shares no code with the CUDA
library (``paper_1902_03317_gb300``) and never imports it.

The arithmetic lives in ``pasta_oracle.c`` (plain C, FP64, single thread, built
with ``gcc -O2 -fno-fast-math``); this module only builds that file, marshals
numpy arrays into it, and adds the mode-order sort, which is a library stable
sort (``numpy.lexsort``) used as one step.

Citations are to arXiv:1902.03317 (PASTA):
  - MTTKRP: Eq. (mttkrp-init) in Sec. 3.6 and Algorithm 6 (Sec. 5.2.6).
  - COO layout and 0-based indices: Sec. 5.1.
  - Row-major factors, element (i, r) at i*R + r: footnote in Sec. 3.4 and
    Algorithm 6.
  - Sorting lexicographically, the first mode most significant: Sec. 5.2.2
    (Algorithm 2's preprocessing); mode orientation: Sec. 2.3.
  - CP model and gradient-descent CPD: Sec. 2.2 (the loss itself is not
    printed in the paper; it is the least-squares objective over the stored
    entries).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pasta_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``pasta_oracle.c`` into ``oracle/_build/liboracle.so`` (and the
    multicore CPU baseline, see ``build_parallel``)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    build_parallel(force)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fno-fast-math", "-ffp-contract=off", "-std=c11",
           "-shared", "-fPIC", "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


_PAR_SRC = os.path.join(_HERE, "pasta_cpu_parallel.c")
_PAR_LIB = os.path.join(_HERE, "_build", "libcpu_parallel.so")
_par = None


def build_parallel(force: bool = False) -> str:
    """Compile the multicore CPU baseline ``pasta_cpu_parallel.c`` (the
    privatization MTTKRP of Sec. 5.3, FP32, OpenMP; a timed baseline, not a
    correctness reference) into ``oracle/_build/libcpu_parallel.so``."""
    os.makedirs(os.path.dirname(_PAR_LIB), exist_ok=True)
    if (not force and os.path.exists(_PAR_LIB)
            and os.path.getmtime(_PAR_LIB) >= os.path.getmtime(_PAR_SRC)):
        return _PAR_LIB
    tmp = _PAR_LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O3", "-fopenmp", "-std=c11", "-shared", "-fPIC", "-o", tmp, _PAR_SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _PAR_LIB)
    return _PAR_LIB


def _load_parallel():
    global _par
    with _lock:
        if _par is None:
            lib = ctypes.CDLL(build_parallel())
            P = ctypes.c_void_p
            lib.cpu_mttkrp_privatized.argtypes = [ctypes.c_int, P, ctypes.c_uint64, P, P, P,
                                                  ctypes.c_int, ctypes.c_int, P, ctypes.c_int]
            lib.cpu_mttkrp_privatized.restype = ctypes.c_int
            lib.cpu_threads.argtypes = []
            lib.cpu_threads.restype = ctypes.c_int
            _par = lib
    return _par


def cpu_threads() -> int:
    """Threads the multicore baseline uses by default (OpenMP's count)."""
    return int(_load_parallel().cpu_threads())


def mttkrp_privatized(dims, idx, val, U, mode: int, threads: int = 0) -> np.ndarray:
    """Mode-``mode`` MTTKRP in FP32 on ``threads`` host threads (0 = all),
    each accumulating a private copy of the output that a parallel pass then
    sums (Sec. 5.3's privatization).  Inputs are converted to FP32 / uint32;
    ``U[mode]`` may be None.  Returns the ``dims[mode] x R`` FP32 output."""
    dims = np.ascontiguousarray(np.asarray(dims, dtype=np.uint64))
    order = int(dims.shape[0])
    idx = [np.ascontiguousarray(np.asarray(ix).astype(np.uint32, copy=False)) for ix in idx]
    val = np.ascontiguousarray(np.asarray(val, dtype=np.float32))
    R = next(np.asarray(u).shape[1] for k, u in enumerate(U) if u is not None and k != mode)
    Uf = [np.zeros((1, R), np.float32) if (u is None or k == mode)
          else np.ascontiguousarray(np.asarray(u, dtype=np.float32)) for k, u in enumerate(U)]
    M = np.empty((int(dims[mode]), R), dtype=np.float32)
    ip = (ctypes.c_void_p * order)(*[_ptr(ix) for ix in idx])
    up = (ctypes.c_void_p * order)(*[_ptr(u) for u in Uf])
    rc = _load_parallel().cpu_mttkrp_privatized(order, _ptr(dims), int(val.shape[0]), ip, _ptr(val), up,
                                                int(mode), int(R), _ptr(M), int(threads))
    if rc != 0:
        raise ValueError("cpu_mttkrp_privatized rejected its arguments or ran out of memory")
    return M


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            for name, argt in {
                "oracle_mttkrp": [ctypes.c_int, P, ctypes.c_uint64, P, P, P,
                                  ctypes.c_int, ctypes.c_int, P],
                "oracle_cp_loss": [ctypes.c_int, P, ctypes.c_uint64, P, P, P,
                                   ctypes.c_int, P, P],
                "oracle_cp_grad": [ctypes.c_int, P, ctypes.c_uint64, P, P, P,
                                   ctypes.c_int, ctypes.c_double, P],
                "oracle_cp_model": [ctypes.c_int, ctypes.c_uint64, P, P, ctypes.c_int, P],
            }.items():
                fn = getattr(lib, name)
                fn.argtypes = argt
                fn.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def _prep(dims, idx, val, U, R):
    dims = np.ascontiguousarray(np.asarray(dims, dtype=np.uint64))
    order = int(dims.shape[0])
    idx = [np.ascontiguousarray(np.asarray(ix).astype(np.uint32, copy=False)) for ix in idx]
    if len(idx) != order:
        raise ValueError("need one index array per mode")
    nnz = int(idx[0].shape[0]) if order else 0
    for ix in idx:
        if ix.shape != (nnz,):
            raise ValueError("index arrays must all have length nnz")
    val = np.ascontiguousarray(np.asarray(val, dtype=np.float64))
    if val.shape != (nnz,):
        raise ValueError("val must have length nnz")
    Ud = []
    for k in range(order):
        if U[k] is None:
            Ud.append(np.zeros((int(dims[k]), R)))
        else:
            u = np.ascontiguousarray(np.asarray(U[k], dtype=np.float64))
            if u.shape != (int(dims[k]), R):
                raise ValueError(f"U[{k}] must be {int(dims[k])} x {R}")
            Ud.append(u)
    idx_ptrs = (ctypes.c_void_p * order)(*[_ptr(ix) for ix in idx])
    u_ptrs = (ctypes.c_void_p * order)(*[_ptr(u) for u in Ud])
    return dims, order, nnz, idx, val, Ud, idx_ptrs, u_ptrs


def mttkrp(dims, idx, val, U, mode: int, R: int | None = None) -> np.ndarray:
    """Mode-``mode`` MTTKRP in FP64: Eq. (mttkrp-init), element-wise as in
    Algorithm 6.  ``U[mode]`` may be ``None``.  Returns ``dims[mode] x R``."""
    if R is None:
        R = next(np.asarray(u).shape[1] for k, u in enumerate(U) if u is not None and k != mode)
    dims, order, nnz, idx, val, Ud, ip, up = _prep(dims, idx, val, U, R)
    M = np.empty((int(dims[mode]), R), dtype=np.float64)
    rc = _load().oracle_mttkrp(order, _ptr(dims), nnz, ip, _ptr(val), up,
                               int(mode), int(R), _ptr(M))
    if rc != 0:
        raise ValueError("oracle_mttkrp rejected its arguments")
    return M


def cp_loss(dims, idx, val, U, want_resid: bool = False):
    """Sparse CP least-squares loss 1/2 sum_m (x_m - sum_r prod_k U_k(i_k,r))^2
    in FP64.  Returns ``loss`` or ``(loss, resid)``."""
    R = int(np.asarray(U[0]).shape[1])
    dims, order, nnz, idx, val, Ud, ip, up = _prep(dims, idx, val, U, R)
    loss = np.zeros(1, dtype=np.float64)
    resid = np.empty(nnz, dtype=np.float64) if want_resid else None
    rc = _load().oracle_cp_loss(order, _ptr(dims), nnz, ip, _ptr(val), up, R,
                                _ptr(resid) if want_resid else None, _ptr(loss))
    if rc != 0:
        raise ValueError("oracle_cp_loss rejected its arguments")
    return (float(loss[0]), resid) if want_resid else float(loss[0])


def cp_model_values(dims, idx, U) -> np.ndarray:
    """CP model sum_r prod_k U_k(i_k(m), r) at every stored coordinate, FP64
    (Sec. 2.2).  Tests also use it to make the values of the planted-model
    workload: ``synth.generate(wl, model_values=...)`` takes this evaluator,
    wrapped by ``planted_model``, since the shared generator holds none of
    the method's arithmetic."""
    R = int(np.asarray(U[0]).shape[1])
    nnz = int(np.asarray(idx[0]).shape[0])
    dims, order, nnz, idx, _, Ud, ip, up = _prep(dims, idx, np.zeros(nnz), U, R)
    out = np.empty(nnz, dtype=np.float64)
    rc = _load().oracle_cp_model(order, nnz, ip, up, R, _ptr(out))
    if rc != 0:
        raise ValueError("oracle_cp_model rejected its arguments")
    return out


def planted_model(coords, planted):
    """``synth.generate``'s ``model_values`` hook backed by the oracle:
    torch coordinates and planted factors in, FP64 torch values out on the
    coordinates' device."""
    import torch
    dims = [int(p.shape[0]) for p in planted]
    v = cp_model_values(dims, [c.cpu().numpy().astype(np.uint32) for c in coords],
                        [p.cpu().double().numpy() for p in planted])
    return torch.from_numpy(v).to(coords[0].device)


def cp_grad(dims, idx, val, U, g: float = 1.0):
    """Gradient of ``g * cp_loss`` with respect to every factor, FP64.
    Returns a list of ``dims[k] x R`` arrays."""
    R = int(np.asarray(U[0]).shape[1])
    dims, order, nnz, idx, val, Ud, ip, up = _prep(dims, idx, val, U, R)
    G = [np.empty((int(dims[k]), R), dtype=np.float64) for k in range(order)]
    gp = (ctypes.c_void_p * order)(*[_ptr(x) for x in G])
    rc = _load().oracle_cp_grad(order, _ptr(dims), nnz, ip, _ptr(val), up, R,
                                float(g), gp)
    if rc != 0:
        raise ValueError("oracle_cp_grad rejected its arguments")
    return G


def mode_order(order: int, mode: int) -> list[int]:
    """Cyclic mode order starting at ``mode``: (n, n+1, ..., N-1, 0, ..., n-1).
    Sec. 5.2.2 sorts lexicographically with the first mode most significant;
    for a mode-n sort the output mode leads and the rest follow cyclically."""
    return [(mode + j) % order for j in range(order)]


def sort_perm(idx, mode: int) -> np.ndarray:
    """Stable lexicographic sort of the stored entries in cyclic mode order
    from ``mode`` (``numpy.lexsort`` as a library step).  Returns the
    permutation p with sorted position q holding original entry p[q]; equal
    coordinates keep their storage order."""
    order = len(idx)
    keys = [np.asarray(idx[k]).astype(np.int64) for k in reversed(mode_order(order, mode))]
    return np.lexsort(keys).astype(np.int64)


# ------------------------------------------------------------------ CP-ALS ---
#
# The paper names alternating least squares as the CPD method and MTTKRP as
# its bottleneck (Sec. 2.2, the CPD paragraph) and cites Kolda and Bader's
# survey for it; the sweep below takes that survey's CP-ALS steps in order:
# for each mode n, V = Hadamard product of U_k^T U_k over k != n, U_n = MTTKRP_n
# times V^{-1}, lambda = the column 2-norms of U_n, and the columns of U_n are
# divided by lambda.  The fit uses ||X - model||^2 = ||X||^2 + ||model||^2 -
# 2 <X, model> with ||X||^2 the sum of the squared stored values (stored
# entries are taken as distinct coordinates).

def gram(U) -> np.ndarray:
    """U^T U in FP64."""
    U = np.asarray(U, dtype=np.float64)
    return U.T @ U


def cp_als_sweep(dims, idx, val, U):
    """One CP-ALS sweep over modes 0..N-1 in FP64.

    Returns ``(U_new, lam, fit)``: the updated factors (columns of unit
    2-norm, a column of zeros staying zero with lambda 0), lambda of the last
    mode, and the fit 1 - ||X - model|| / ||X|| of the model sum_r lam_r
    U_0(:, r) o ... o U_{N-1}(:, r).  A singular V raises
    ``numpy.linalg.LinAlgError``."""
    N = len(dims)
    U = [np.array(u, dtype=np.float64, copy=True) for u in U]
    R = U[0].shape[1]
    G = [gram(u) for u in U]
    lam = np.ones(R)
    M = None
    for n in range(N):
        M = mttkrp(dims, idx, val, U, n, R)
        V = np.ones((R, R))
        for k in range(N):
            if k != n:
                V *= G[k]
        # U_n = M V^{-1}; V is symmetric, so solve V U_n^T = M^T
        Un = np.linalg.solve(V, M.T).T
        lam = np.sqrt(np.sum(Un * Un, axis=0))
        inv = np.where(lam > 0, 1.0 / np.where(lam > 0, lam, 1.0), 0.0)
        U[n] = Un * inv[None, :]
        G[n] = gram(U[n])
    fit = cp_fit(val, U, lam, M)
    return U, lam, fit


def cp_fit(val, U, lam, M_last) -> float:
    """Fit of the model (lam; U) to the stored entries, given the MTTKRP of
    the last mode computed from the other (final) factors:
    <X, model> = sum_r lam_r sum_i M_last(i, r) U_{N-1}(i, r) and
    ||model||^2 = lam^T (Hadamard over k of U_k^T U_k) lam."""
    val = np.asarray(val, dtype=np.float64)
    normx2 = float(np.dot(val, val))
    H = np.ones((lam.shape[0], lam.shape[0]))
    for u in U:
        H *= gram(u)
    norm_model2 = float(lam @ H @ lam)
    inner = float(np.sum(lam * np.sum(np.asarray(M_last) * U[-1], axis=0)))
    res2 = max(normx2 + norm_model2 - 2.0 * inner, 0.0)
    return 1.0 - np.sqrt(res2) / np.sqrt(normx2) if normx2 > 0 else 0.0


# ------------------------------------------------------------ TEW-eq, TS ---
#
# Element-wise operations between two tensors with the same coordinates
# (TEW-eq, Sec. 3.1 and Algorithm 1) and between a tensor and a scalar (TS,
# Sec. 3.2 and Algorithm 3).  The coordinates pass through unchanged; only the
# values are combined.  FP64 arithmetic on the (FP32) stored values; the GPU
# computes in FP32, so parity is stated in FP32 units in the last place.

OPS = ("add", "sub", "mul", "div")


def _apply(op: str, a, b):
    if op == "add":
        return a + b
    if op == "sub":
        return a - b
    if op == "mul":
        return a * b
    if op == "div":
        with np.errstate(divide="ignore", invalid="ignore"):
            return a / b
    raise ValueError(f"unknown op {op!r}")


def tew_eq(idx_x, val_x, idx_y, val_y, op: str):
    """Z = X op Y for tensors with identical coordinate lists (Algorithm 1).
    Returns (idx_z, val_z) in FP64; raises if the coordinates differ."""
    for a, b in zip(idx_x, idx_y):
        if not np.array_equal(np.asarray(a), np.asarray(b)):
            raise ValueError("TEW-eq needs the same coordinates in the same order")
    vx = np.asarray(val_x, dtype=np.float64)
    vy = np.asarray(val_y, dtype=np.float64)
    return [np.asarray(a).copy() for a in idx_x], _apply(op, vx, vy)


def ts(idx_x, val_x, op: str, s: float):
    """Y = X op s for every stored entry (Algorithm 3 for multiplication;
    the other operators alike).  Returns (idx_y, val_y) in FP64."""
    vx = np.asarray(val_x, dtype=np.float64)
    return [np.asarray(a).copy() for a in idx_x], _apply(op, vx, np.float64(s))


# -------------------------------------------------------------- TTV, TTM ---
#
# Mode-n products (Sec. 3.3 and 3.4, Algorithms 4 and 5).  The result keeps
# one entry per mode-n fiber of X (the stored entries sharing every index but
# i_n), Y(f, r) = sum over the fiber's entries of x * U(i_n, r) (TTV: R = 1,
# U = v).  Fibers are listed in lexicographic order of their coordinates in
# the cyclic mode order n+1, ..., N-1, 0, ..., n-1 (numpy.lexsort as a library
# step), the order in which the mode-(n+1) sorted copy holds them.

def fiber_modes(order: int, mode: int) -> list[int]:
    """The modes of a mode-n fiber's coordinates, in cyclic order from n+1."""
    return [(mode + j) % order for j in range(1, order)]


def ttm(dims, idx, val, U, mode: int):
    """Y = X x_n U with U of shape dims[mode] x R (the paper's transposed
    convention).  Returns (fiber_coords: list of N-1 uint32 arrays, in the
    modes of fiber_modes(), Y: nfibs x R FP64)."""
    N = len(dims)
    U = np.asarray(U, dtype=np.float64)
    if U.ndim == 1:
        U = U[:, None]
    modes = fiber_modes(N, mode)
    idx = [np.asarray(ix).astype(np.int64) for ix in idx]
    val = np.asarray(val, dtype=np.float64)
    acc: dict[tuple, np.ndarray] = {}
    for m in range(val.shape[0]):
        key = tuple(int(idx[k][m]) for k in modes)
        row = acc.get(key)
        if row is None:
            row = np.zeros(U.shape[1])
            acc[key] = row
        row += val[m] * U[int(idx[mode][m])]
    keys = list(acc.keys())
    if not keys:
        return [np.zeros(0, dtype=np.uint32) for _ in modes], np.zeros((0, U.shape[1]))
    K = np.array(keys, dtype=np.int64)
    order = np.lexsort(K.T[::-1])
    coords = [K[order, j].astype(np.uint32) for j in range(len(modes))]
    Y = np.stack([acc[keys[i]] for i in order])
    return coords, Y


def ttv(dims, idx, val, v, mode: int):
    """Y = X x_n v (Algorithm 4): TTM with a single column.  Returns
    (fiber_coords, y with one value per fiber)."""
    coords, Y = ttm(dims, idx, val, np.asarray(v, dtype=np.float64)[:, None], mode)
    return coords, Y[:, 0]


def hicoo(dims, idx, val, bits: int):
    """The HiCOO copy (Li, Choi and Vuduc, SC'18; Sec. 8 names it as a format
    to add) from its definition: blocks of 2^bits cells per mode; an entry's
    block coordinate is i_k >> bits, its offset i_k & (2^bits - 1).  Entries
    are ordered by one stable sort of the key made of the block coordinates
    (mode 0 most significant, each mode ceil(log2(number of blocks)) bits)
    followed by the offsets (mode 0 first, bits each), cut to its leading 64
    bits (numpy's stable argsort as the sorting step).  Returns
    (bptr [nb + 1], binds: N arrays [nb], einds: N arrays [nnz] (uint8),
    val [nnz], perm [nnz]: creation-order entry of each position)."""
    dims = [int(d) for d in dims]
    N = len(dims)
    idx = [np.asarray(i, dtype=np.uint64) for i in idx]
    nnz = int(idx[0].shape[0]) if N else 0
    bb = []
    for d in dims:
        nblk = (d + (1 << bits) - 1) >> bits
        bb.append(int(nblk - 1).bit_length())
    BB = sum(bb)
    if BB > 64:
        raise ValueError("block coordinates need more than 64 key bits")
    E = min(64 - BB, N * bits)
    block_key = np.zeros(nnz, dtype=np.uint64)
    elem_key = np.zeros(nnz, dtype=np.uint64)
    mask = np.uint64((1 << bits) - 1)
    for k in range(N):
        block_key = (block_key << np.uint64(bb[k])) | (idx[k] >> np.uint64(bits))
        elem_key = (elem_key << np.uint64(bits)) | (idx[k] & mask)
    drop = N * bits - E
    e_part = elem_key >> np.uint64(drop) if drop < 64 else np.zeros(nnz, dtype=np.uint64)
    key = (block_key << np.uint64(E)) | e_part if E < 64 else e_part
    perm = np.argsort(key, kind="stable")
    bk = block_key[perm]
    heads = np.ones(nnz, dtype=bool)
    if nnz:
        heads[1:] = bk[1:] != bk[:-1]
    starts = np.flatnonzero(heads)
    bptr = np.concatenate([starts, [nnz]]).astype(np.int64)
    binds = [(idx[k][perm][starts] >> np.uint64(bits)).astype(np.int64) for k in range(N)]
    einds = [(idx[k][perm] & mask).astype(np.uint8) for k in range(N)]
    return bptr, binds, einds, np.asarray(val)[perm], perm
