"""Pins of the oracle's HiCOO copy (oracle.hicoo), CPU only.

- a hand-worked 4 x 4 x 3 example with 2 x 2 x 2 blocks (tests/golden);
- the copy is a reordering: block coordinates and offsets rebuild the sorted
  coordinates, and the values follow;
- blocks strictly increase in lexicographic order, every entry lies in its
  block's window, offsets inside a block are in lexicographic order (no key
  cut) and a block's entries are contiguous;
- MTTKRP of the rebuilt tensor equals MTTKRP of the original (Eq.
  (mttkrp-init) does not depend on storage order);
- with a key cut (block bits plus offset bits above 64), entries with equal
  leading bits keep creation order;
- planted mistakes (offsets before blocks, reversed mode order) fail a pin.
"""
import os

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _golden():
    data, ent, in_e = {}, [], False
    for line in open(os.path.join(ROOT, "tests", "golden", "hicoo_4x4x3.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if ":" in line:
            k, rest = line.split(":", 1)
            in_e = k.strip() == "entries"
            if not in_e:
                data[k.strip()] = [int(float(x)) for x in rest.split()]
        elif in_e:
            ent.append([int(x) for x in line.split()])
    ent = np.array(ent)
    return data, [ent[:, k].astype(np.uint32) for k in range(3)], ent[:, 3].astype(np.float64)


def test_golden_4x4x3():
    g, idx, val = _golden()
    bptr, binds, einds, v, perm = oracle.hicoo(g["dims"], idx, val, g["bits"][0])
    assert bptr.tolist() == g["bptr"]
    for k in range(3):
        assert binds[k].tolist() == g[f"binds{k}"]
        assert einds[k].tolist() == g[f"einds{k}"]
    assert v.tolist() == g["val"]


def _rebuild(bptr, binds, einds, bits):
    nb = len(bptr) - 1
    blk = np.repeat(np.arange(nb), np.diff(bptr))
    return [(binds[k][blk] << bits) + einds[k].astype(np.int64) for k in range(len(binds))]


@pytest.mark.parametrize("dims,bits", [((40, 30, 20), 2), ((300, 200, 100, 7), 3), ((9, 1000, 500), 7),
                                       ((5, 6, 7, 8, 9), 1)])
def test_reordering_and_block_structure(dims, bits):
    rng = np.random.default_rng(len(dims) * 10 + bits)
    nnz = 4000
    idx = [rng.integers(0, d, nnz).astype(np.uint32) for d in dims]
    idx[0][:50] = idx[0][50:100]  # a few duplicates of other coordinates
    for k in range(1, len(dims)):
        idx[k][:50] = idx[k][50:100]
    val = rng.standard_normal(nnz)
    bptr, binds, einds, v, perm = oracle.hicoo(dims, idx, val, bits)
    coords = _rebuild(bptr, binds, einds, bits)
    for k in range(len(dims)):
        assert np.array_equal(coords[k], idx[k][perm].astype(np.int64))
    assert np.array_equal(v, val[perm])
    assert sorted(perm.tolist()) == list(range(nnz))
    # blocks strictly increasing (lexicographic), offsets ordered inside a block
    btup = list(zip(*[b.tolist() for b in binds]))
    assert all(a < b for a, b in zip(btup, btup[1:]))
    for b in range(len(bptr) - 1):
        lo, hi = bptr[b], bptr[b + 1]
        assert hi > lo
        et = list(zip(*[e[lo:hi].tolist() for e in einds]))
        assert et == sorted(et)
        for k in range(len(dims)):
            assert np.all(coords[k][lo:hi] >> bits == binds[k][b])


def test_mttkrp_of_the_copy():
    rng = np.random.default_rng(3)
    dims = (60, 50, 40, 6)
    nnz = 3000
    idx = [rng.integers(0, d, nnz).astype(np.uint32) for d in dims]
    val = rng.standard_normal(nnz)
    U = [rng.standard_normal((d, 5)) for d in dims]
    bptr, binds, einds, v, _ = oracle.hicoo(dims, idx, val, 3)
    coords = [c.astype(np.uint32) for c in _rebuild(bptr, binds, einds, 3)]
    for n in range(4):
        a = oracle.mttkrp(dims, coords, v, U, n)
        b = oracle.mttkrp(dims, idx, val, U, n)
        assert np.allclose(a, b, rtol=1e-12, atol=1e-12)


def test_key_cut_keeps_creation_order():
    # 2^22-sized modes with 1-bit blocks: 3 x 21 block bits leave one offset
    # bit of the three, so entries differing only in the last two offsets
    # keep creation order
    dims = (1 << 22, 1 << 22, 1 << 22)
    idx = [np.array([6, 6, 6, 6], np.uint32), np.array([9, 9, 8, 9], np.uint32),
           np.array([5, 4, 4, 4], np.uint32)]
    val = np.arange(4.0)
    bptr, binds, einds, v, perm = oracle.hicoo(dims, idx, val, 1)
    # blocks (3,4,2) holds m0, m1, m3 ((9,5), (9,4), (9,4)); (3,4,2) vs m2 (8,4): same block
    assert len(bptr) == 2
    assert perm.tolist() == [0, 1, 2, 3]  # offset bit of mode 0 equal; the rest cut


def test_planted_mistakes_fail():
    g, idx, val = _golden()

    def offsets_first(dims, idx, val, bits):
        key = [((i & ((1 << bits) - 1)).astype(np.int64) << 8) + (i >> bits).astype(np.int64) for i in idx]
        return np.lexsort(key[::-1])

    def reversed_modes(dims, idx, val, bits):
        return oracle.hicoo(dims[::-1], idx[::-1], val, bits)[4]

    want = oracle.hicoo(g["dims"], idx, val, 1)[4]
    assert not np.array_equal(offsets_first(g["dims"], idx, val, 1), want)
    assert not np.array_equal(reversed_modes(g["dims"], idx, val, 1), want)
