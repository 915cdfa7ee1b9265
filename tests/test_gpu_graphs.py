"""The hot path under CUDA-graph capture: MTTKRP on every mode and the fused
loss with every gradient are enqueued on the capturing stream only (no
allocation, no synchronisation inside), so a captured step replays them.
Replays must give the eager results (same kernels, same launch shapes; the
loss is bit-reproducible, the FP32 atomics are compared at the MTTKRP bar)."""
import pytest
import torch

import paper_1902_03317_gb300 as pasta
from paper_1902_03317_gb300 import synth
from tests import _gpu as G

pytestmark = pytest.mark.gpu


def test_captured_step_replays_eager_results():
    wl = G.small("zipf3d", 200_001, (5_000, 3_000, 2_000))
    Xh = synth.generate(wl)
    X = G.to_device(Xh)
    X.sort_all()
    Us = [u.to(G.DEV).contiguous() for u in synth.generate_factors(wl.dims, wl.R, seed=5)]
    Ms = [torch.empty((d, wl.R), device=G.DEV) for d in wl.dims]

    def step():
        for n in range(3):
            pasta.mttkrp(X, Us, n, out=Ms[n])
        return pasta.cp_loss_fwd_bwd(X, Us)

    loss_e, grads_e = step()
    Ms_e = [m.clone() for m in Ms]
    torch.cuda.synchronize()

    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):  # warm up on the side stream before capture
        step()
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        loss_g, grads_g = step()
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    assert float(loss_g) == float(loss_e)  # fixed-order FP64 reduction
    for a, b in zip(grads_g, grads_e):
        assert G.rel_err(a.cpu().numpy(), b.cpu().numpy()) < G.FP32_TOL
    for a, b in zip(Ms, Ms_e):
        assert G.rel_err(a.cpu().numpy(), b.cpu().numpy()) < G.FP32_TOL
    X.close()
