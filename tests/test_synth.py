"""Seeded input generators (CPU): sizes, bounds, distinctness, skew, seeding."""
import numpy as np
import torch

from paper_1902_03317_gb300 import synth


def test_distinct_uniform_exact_nnz_and_bounds():
    wl = synth.WORKLOADS["uniform3d_200"]
    X = synth.generate(wl)
    assert X.nnz == wl.nnz
    keys = set()
    for m in range(0, X.nnz, 7):
        keys.add(tuple(int(ix[m]) for ix in X.idx))
    for k, ix in enumerate(X.idx):
        assert ix.dtype == torch.int32
        assert int(ix.min()) >= 0 and int(ix.max()) < wl.dims[k]
    packed = synth._pack(X.idx, wl.dims)
    assert torch.unique(packed).numel() == wl.nnz
    assert float(X.val.min()) >= -1.0 and float(X.val.max()) <= 1.0


def test_zipf_distinct_small_is_skewed_and_distinct():
    wl = synth.WORKLOADS["zipf3d"].scaled(nnz=50_000, dims=(5000, 2500, 1000))
    X = synth.generate(wl)
    assert X.nnz == 50_000
    assert torch.unique(synth._pack(X.idx, wl.dims)).numel() == 50_000
    counts = np.bincount(X.idx[0].numpy(), minlength=5000)
    # heavy head: the largest slice holds far more than the mean
    assert counts.max() > 20 * counts.mean()
    assert float(X.val.min()) > 0


def test_duplicates_kept_when_not_distinct():
    wl = synth.WORKLOADS["zipf4d"].scaled(nnz=20_000, dims=(500, 500, 50, 10))
    X = synth.generate(wl)
    assert X.nnz == 20_000
    assert torch.unique(synth._pack(X.idx, wl.dims)).numel() < 20_000


def test_seeded_reproducible_and_seed_sensitive():
    wl = synth.WORKLOADS["zipf5d"].scaled(nnz=4096, dims=(8, 1000, 500, 100, 10))
    a = synth.generate(wl)
    b = synth.generate(wl)
    c = synth.generate(wl, seed=99)
    for x, y in zip(a.idx, b.idx):
        assert torch.equal(x, y)
    assert torch.equal(a.val, b.val)
    assert not torch.equal(a.idx[1], c.idx[1])
    assert int(a.idx[0].max()) < 8


def test_planted_values_are_model_plus_noise():
    """The generator asks the caller for the planted model's values and adds
    N(0, sigma^2) noise; a planted workload without an evaluator is refused."""
    import pytest
    wl = synth.WORKLOADS["cploss3d"].scaled(nnz=3000, dims=(40, 40, 40))
    with pytest.raises(ValueError):
        synth.generate(wl)
    seen = {}

    def fixed(coords, planted):
        seen["shapes"] = ([tuple(c.shape) for c in coords], [tuple(p.shape) for p in planted])
        return torch.full((coords[0].numel(),), 3.0, dtype=torch.float64)

    X = synth.generate(wl, model_values=fixed)
    assert seen["shapes"] == ([(3000,)] * 3, [(40, 16)] * 3)
    assert X.planted is not None and X.planted[0].shape == (40, 16)
    noise = (X.val - 3.0).double()
    assert abs(float(noise.mean())) < 2e-3
    assert 0.009 < float(noise.std()) < 0.011
