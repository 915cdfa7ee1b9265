"""The library's device buffers go through torch's caching allocator
(pasta_set_allocator): visible in torch's accounting, returned on destroy,
and the allocator cannot be swapped while library buffers are held."""
import gc

import pytest
import torch

import paper_1902_03317_gb300 as pasta
from paper_1902_03317_gb300 import synth
from tests import _gpu as G

pytestmark = pytest.mark.gpu


def test_buffers_come_from_torch_and_go_back():
    gc.collect()
    wl = G.small("zipf3d", 200_000, (3_000, 2_000, 1_000))
    Xh = synth.generate(wl)
    idx = [i.to(G.DEV) for i in Xh.idx]
    val = Xh.val.to(G.DEV)
    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated()
    X = pasta.CooTensor(wl.dims, idx, val)
    X.sort_all()
    held = torch.cuda.memory_allocated() - before
    # creation-order copy (N + 1 arrays) + three sorted copies (N + 2 arrays), padded
    assert held >= 200_000 * 4 * ((3 + 1) + 3 * (3 + 2))
    with pytest.raises(pasta.PastaError):
        pasta.use_torch_allocator(False)  # blocks are held
    X.close()
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == before
    pasta.use_torch_allocator(False)
    Y = pasta.CooTensor(wl.dims, idx, val)
    assert torch.cuda.memory_allocated() == before  # cudaMalloc: not torch's
    Y.close()
    pasta.use_torch_allocator(True)
