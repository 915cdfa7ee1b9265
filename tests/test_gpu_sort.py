"""Mode-order sort (Sec. 5.2.2) on the GPU vs the oracle's stable lexsort.

Where the packed key holds every mode (at most 64 bits), the stable sort is
unique and the permutation must match bit for bit.  Where the key is cut to
its leading 64 bits, only the order of the fully included modes is fixed:
that part is compared, the rest is checked to be a valid permutation.
"""
import numpy as np
import pytest
import torch

import oracle
from tests import _gpu as G

pytestmark = pytest.mark.gpu


CASES = [
    ("uniform3d_200", 20_000, (200, 200, 200)),
    ("zipf3d", 50_000, (5000, 3000, 1000)),
    ("zipf4d", 60_000, (3000, 3000, 300, 60)),      # duplicates kept
    ("zipf5d", 40_000, (8, 2000, 500, 100, 10)),    # duplicates kept
]


@pytest.mark.parametrize("name,nnz,dims", CASES)
def test_sorted_copies_match_oracle_exactly(name, nnz, dims):
    Xh = G.generate(G.small(name, nnz, dims))
    idx, val = G.host(Xh)
    X = G.to_device(Xh)
    for mode in range(len(dims)):
        X.sort_by_mode(mode)
        sidx, sval, perm = X.copy_out(mode)
        perm = perm.cpu().numpy().astype(np.int64)
        np.testing.assert_array_equal(perm, oracle.sort_perm(idx, mode))
        for k in range(len(dims)):
            np.testing.assert_array_equal(sidx[k].cpu().numpy().astype(np.uint32), idx[k][perm])
        np.testing.assert_array_equal(sval.cpu().numpy(), val[perm].astype(np.float32))
    # the creation-order copy is untouched
    oidx, oval, _ = X.copy_out(-1)
    np.testing.assert_array_equal(oidx[1].cpu().numpy().astype(np.uint32), idx[1])
    X.close()


@pytest.mark.parametrize("name,nnz,dims", CASES[:3])
def test_sort_order_independent_of_which_copies_exist(name, nnz, dims):
    """A mode's copy may be sorted from the next mode's copy on its own field
    alone, or from the previous mode's copy on the other fields; the result
    must equal the sort from the creation order whatever was sorted before."""
    Xh = G.generate(G.small(name, nnz, dims))
    idx, val = G.host(Xh)
    N = len(dims)
    for sequence in (list(reversed(range(N))), [1, 0] + list(range(2, N)), [0] + list(range(N - 1, 0, -1)),
                     [N - 1, 0] + list(range(1, N - 1))):
        X = G.to_device(Xh)
        for mode in sequence:
            X.sort_by_mode(mode)
        for mode in range(N):
            sidx, sval, perm = X.copy_out(mode)
            perm = perm.cpu().numpy().astype(np.int64)
            np.testing.assert_array_equal(perm, oracle.sort_perm(idx, mode))
            for k in range(N):
                np.testing.assert_array_equal(sidx[k].cpu().numpy().astype(np.uint32), idx[k][perm])
            np.testing.assert_array_equal(sval.cpu().numpy(), val[perm].astype(np.float32))
        X.close()


def test_key_cut_to_64_bits_keeps_leading_modes_sorted():
    # 3 + 24 + 21 + 17 + 10 = 75 bits: the key holds modes 0,1,2 and the top
    # 16 bits of mode 3 when sorting for mode 0.
    dims = (8, 10_000_000, 2_000_000, 100_000, 1_000)
    Xh = G.generate(G.small("zipf5d", 30_000, dims))
    idx, _ = G.host(Xh)
    X = G.to_device(Xh)
    for mode in range(5):
        X.sort_by_mode(mode)
        _, _, perm = X.copy_out(mode)
        perm = perm.cpu().numpy().astype(np.int64)
        assert np.array_equal(np.sort(perm), np.arange(perm.size))
        order = oracle.mode_order(5, mode)
        bits = [max(0, int(dims[k] - 1).bit_length()) for k in order]
        full = []
        used = 0
        for k, b in zip(order, bits):
            if used + b > 64:
                break
            full.append(k)
            used += b
        # the leading fully-included modes are in lexicographic order
        keys = np.stack([idx[k][perm].astype(np.int64) for k in full], axis=1)
        lex = np.lexsort(keys.T[::-1])
        assert np.array_equal(lex, np.arange(perm.size)), f"mode {mode} not sorted"
        np.testing.assert_array_equal(idx[mode][perm], np.sort(idx[mode]))
    X.close()


@pytest.mark.parametrize("nnz", [0, 1, 2, 5, 4095, 4096, 4097])
def test_sort_small_and_ragged(nnz):
    dims = (7, 5, 3)
    g = torch.Generator().manual_seed(nnz)
    Xh = G.synth.Tensor(None, dims, [torch.randint(0, d, (nnz,), generator=g, dtype=torch.int32) for d in dims],
                        torch.rand(nnz, generator=g))
    idx, _ = G.host(Xh)
    X = G.to_device(Xh)
    for mode in range(3):
        X.sort_by_mode(mode)
        _, _, perm = X.copy_out(mode)
        np.testing.assert_array_equal(perm.cpu().numpy().astype(np.int64), oracle.sort_perm(idx, mode))
    X.close()


@pytest.mark.parametrize("dims", [(5, 1, 1), (1, 1, 1), (1, 6, 1, 3)])
def test_sort_with_size_one_modes(dims):
    """Modes of size 1 take no key bits; a copy derived from the previous
    mode's copy can then have no bit left to sort (one pass of width 0)."""
    nnz = 3000
    g = torch.Generator().manual_seed(len(dims) + sum(dims))
    Xh = G.synth.Tensor(None, dims, [torch.randint(0, d, (nnz,), generator=g, dtype=torch.int32) for d in dims],
                        torch.rand(nnz, generator=g))
    idx, val = G.host(Xh)
    N = len(dims)
    for sequence in (list(range(N)), list(reversed(range(N)))):
        X = G.to_device(Xh)
        for mode in sequence:
            X.sort_by_mode(mode)
        for mode in range(N):
            sidx, sval, perm = X.copy_out(mode)
            perm = perm.cpu().numpy().astype(np.int64)
            np.testing.assert_array_equal(perm, oracle.sort_perm(idx, mode))
            for k in range(N):
                np.testing.assert_array_equal(sidx[k].cpu().numpy().astype(np.uint32), idx[k][perm])
            np.testing.assert_array_equal(sval.cpu().numpy(), val[perm].astype(np.float32))
        X.close()


@pytest.mark.parametrize("pinned", [True, False])
def test_create_from_host_memory(pinned):
    """pasta_coo_create takes host pointers too (copied with cudaMemcpyDefault):
    the creation-order and sorted copies match a handle created from device
    memory bit for bit, and so does the MTTKRP up to the order of the
    tile-edge atomic additions."""
    Xh = G.generate(G.small("zipf3d", 30_001, (3_000, 2_000, 1_000)))
    idx_h = [i.contiguous() for i in Xh.idx]
    val_h = Xh.val.contiguous()
    if pinned:
        idx_h = [i.pin_memory() for i in idx_h]
        val_h = val_h.pin_memory()
    Xa = G.pasta.CooTensor(Xh.dims, idx_h, val_h, device=G.DEV)
    Xb = G.to_device(Xh)
    oa, va, _ = Xa.copy_out(-1)
    for k in range(3):
        assert torch.equal(oa[k].cpu(), Xh.idx[k])
    assert torch.equal(va.cpu(), Xh.val)
    _, dev_u, _ = G.factors(Xh.dims, 16, 5)
    for n in range(3):
        Ma, Mb = G.pasta.mttkrp(Xa, dev_u, n), G.pasta.mttkrp(Xb, dev_u, n)
        assert G.rel_err(Ma.cpu().numpy(), Mb.cpu().numpy()) < 1e-6
        sa, sva, pa = Xa.copy_out(n)
        sb, svb, pb = Xb.copy_out(n)
        assert torch.equal(pa, pb) and torch.equal(sva, svb)
        assert all(torch.equal(x, y) for x, y in zip(sa, sb))
    Xa.close()
    Xb.close()


@pytest.mark.parametrize("nbytes", [4, 12, 16, 4100, 1 << 20, (1 << 20) + 12])
def test_memcpy_every_direction(nbytes):
    """pasta_memcpy (copy_): pinned host -> device, device -> pinned host,
    device -> device and pageable host -> device, bit for bit, at sizes with
    and without a ragged tail of words."""
    n = nbytes // 4
    g = torch.Generator().manual_seed(nbytes)
    h = torch.randint(-2**31, 2**31 - 1, (n,), generator=g, dtype=torch.int32)
    hp = h.pin_memory()
    d = torch.empty(n, dtype=torch.int32, device=G.DEV)
    G.pasta.copy_(d, hp)
    torch.cuda.synchronize()
    assert torch.equal(d.cpu(), h)
    back = torch.zeros(n, dtype=torch.int32).pin_memory()
    G.pasta.copy_(back, d)
    torch.cuda.synchronize()
    assert torch.equal(back, h)
    d2 = torch.empty_like(d)
    G.pasta.copy_(d2, d)
    d3 = torch.empty_like(d)
    G.pasta.copy_(d3, h)  # pageable source
    torch.cuda.synchronize()
    assert torch.equal(d2.cpu(), h) and torch.equal(d3.cpu(), h)
    # an offset view (4-byte aligned, not 16): the copy-engine path; a
    # 16-byte aligned interior view of the pinned block: the kernel path
    if n > 2:
        G.pasta.copy_(d[1:], hp[1:])
        torch.cuda.synchronize()
        assert torch.equal(d.cpu(), h)
    if n > 4:
        d.zero_()
        G.pasta.copy_(d[4:], hp[4:])
        back.zero_()
        G.pasta.copy_(back[4:], d[4:])
        torch.cuda.synchronize()
        assert torch.equal(d[4:].cpu(), h[4:]) and torch.equal(back[4:], h[4:])


@pytest.mark.parametrize("name,nnz,dims,mode", [
    ("zipf3d", 5_000_003, (200_000, 100_000, 40_000), 0),
    ("zipf4d", 4_500_001, (50_000, 50_000, 5_000, 1_000), 2),   # duplicates kept, odd halves
    ("zipf3d", 17_000_001, (400_000, 200_000, 80_000), 1),      # larger halves, another mode
])
def test_create_sorted_overlapped_matches_oracle(name, nnz, dims, mode):
    """pasta_coo_create_sorted from pinned host arrays (>= 2^22 entries: the
    first half sorted while the second is copied in, then merged) gives the
    oracle's permutation and sorted copy bit for bit, and the creation-order
    copy unchanged; the other modes sort from it as usual."""
    Xh = G.generate(G.small(name, nnz, dims))
    idx, val = G.host(Xh)
    idx_h = [i.contiguous().pin_memory() for i in Xh.idx]
    val_h = Xh.val.contiguous().pin_memory()
    X = G.pasta.CooTensor(Xh.dims, idx_h, val_h, device=G.DEV, sort_mode=mode)
    sidx, sval, perm = X.copy_out(mode)
    perm = perm.cpu().numpy().astype(np.int64)
    np.testing.assert_array_equal(perm, oracle.sort_perm(idx, mode))
    for k in range(len(dims)):
        np.testing.assert_array_equal(sidx[k].cpu().numpy().astype(np.uint32), idx[k][perm])
    np.testing.assert_array_equal(sval.cpu().numpy(), val[perm].astype(np.float32))
    oidx, oval, _ = X.copy_out(-1)
    for k in range(len(dims)):
        assert torch.equal(oidx[k].cpu(), Xh.idx[k])
    assert torch.equal(oval.cpu(), Xh.val)
    nxt = (mode + len(dims) - 1) % len(dims)
    X.sort_by_mode(nxt)
    _, _, p2 = X.copy_out(nxt)
    np.testing.assert_array_equal(p2.cpu().numpy().astype(np.int64), oracle.sort_perm(idx, nxt))
    X.close()


def test_create_sorted_fallbacks_and_errors():
    """Below 2^22 entries, or from device memory, create_sorted runs create
    and sort; a mode outside [0, order) is refused."""
    Xh = G.generate(G.small("zipf3d", 30_001, (3_000, 2_000, 1_000)))
    idx, _ = G.host(Xh)
    for X in (G.pasta.CooTensor(Xh.dims, [i.pin_memory() for i in Xh.idx], Xh.val.pin_memory(),
                                device=G.DEV, sort_mode=1),
              G.pasta.CooTensor(Xh.dims, [i.to(G.DEV) for i in Xh.idx], Xh.val.to(G.DEV), sort_mode=1)):
        _, _, perm = X.copy_out(1)
        np.testing.assert_array_equal(perm.cpu().numpy().astype(np.int64), oracle.sort_perm(idx, 1))
        X.close()
    with pytest.raises(G.pasta.PastaError):
        G.pasta.CooTensor(Xh.dims, [i.to(G.DEV) for i in Xh.idx], Xh.val.to(G.DEV), sort_mode=3)


def test_create_sorted_large_cut_key_falls_back():
    """At >= 2^22 pinned entries but with a key cut at 64 bits (zipf5d's 75
    bits), create_sorted takes the create-then-sort path: its copy equals the
    one a separate create and sort give, bit for bit."""
    dims = (8, 10_000_000, 2_000_000, 100_000, 1_000)
    Xh = G.generate(G.small("zipf5d", 4_200_000, dims))
    idx_h = [i.contiguous().pin_memory() for i in Xh.idx]
    val_h = Xh.val.contiguous().pin_memory()
    A = G.pasta.CooTensor(Xh.dims, idx_h, val_h, device=G.DEV, sort_mode=1)
    B = G.to_device(Xh)
    B.sort_by_mode(1)
    ia, va, pa = A.copy_out(1)
    ib, vb, pb = B.copy_out(1)
    assert torch.equal(pa, pb) and torch.equal(va, vb)
    assert all(torch.equal(x, y) for x, y in zip(ia, ib))
    A.close()
    B.close()
