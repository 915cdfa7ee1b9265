"""pasta_gather_probe: the row gathers of the streaming MTTKRP without its
arithmetic.  The sum of everything it wrote must be the sum, over the stored
entries, of every element of the N-1 rows MTTKRP gathers for the mode, so the
probe cannot skip gathers; checked against that sum in FP64, to 1e-5 of the
sum of the magnitudes (the probe adds in FP32)."""
import numpy as np
import pytest
import torch

import paper_1902_03317_gb300 as pasta
from tests import _gpu as G

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name,nnz,dims,R,dtype", [
    ("zipf3d", 200_000, (20_000, 10_000, 4_000), 32, torch.float32),
    ("zipf4d", 100_000, (3_000, 3_000, 300, 60), 64, torch.bfloat16),
    ("zipf5d", 150_000, (8, 50_000, 10_000, 1_000, 100), 16, torch.float32),
])
def test_gather_probe_sums_the_gathered_rows(name, nnz, dims, R, dtype):
    Xh = G.generate(G.small(name, nnz, dims))
    idx, _ = G.host(Xh)
    _, dev, rounded = G.factors(dims, R, 41, dtype)
    X = G.to_device(Xh)
    for n in range(len(dims)):
        sink = torch.zeros(1 << 20, dtype=torch.float32, device=G.DEV)
        pasta.gather_probe(X, dev, n, sink=sink)
        got = float(sink.double().sum())
        others = [k for k in range(len(dims)) if k != n]
        want = sum(float(rounded[k].sum(axis=1)[idx[k].astype(np.int64)].sum()) for k in others)
        scale = sum(float(np.abs(rounded[k]).sum(axis=1)[idx[k].astype(np.int64)].sum()) for k in others)
        assert abs(got - want) <= 1e-5 * scale, (n, got, want, scale)
    X.close()


def test_gather_probe_rejects_uncovered_cases():
    Xh = G.generate(G.small("zipf3d", 1000, (50, 40, 30)))
    X = G.to_device(Xh)
    _, dev, _ = G.factors((50, 40, 30), 5, 1)  # R = 5: not a streaming case
    with pytest.raises(pasta.PastaError) as e:
        pasta.gather_probe(X, dev, 0)
    assert e.value.name == "PASTA_ERR_UNSUPPORTED"
    X.close()
