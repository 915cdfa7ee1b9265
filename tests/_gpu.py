"""Helpers shared by the GPU parity tests."""
from __future__ import annotations

import numpy as np
import torch

import oracle
import paper_1902_03317_gb300 as pasta
from paper_1902_03317_gb300 import synth

DEV = "cuda:0"
FP32_TOL = 1e-5   # rel. Frobenius, FP32 factors, vs the FP64 oracle
LOWP_TOL = 1e-2   # rel. Frobenius, BF16/FP16 factors, end to end vs FP32 master factors


def rel_err(a, b) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = float(np.linalg.norm(b))
    return float(np.linalg.norm(a - b)) / (nb if nb > 0 else 1.0)


def host(Xh: synth.Tensor):
    """numpy views of a generated tensor for the oracle."""
    return ([i.cpu().numpy().astype(np.uint32) for i in Xh.idx],
            Xh.val.cpu().numpy().astype(np.float64))


def to_device(Xh: synth.Tensor, validate: bool = True) -> pasta.CooTensor:
    return pasta.CooTensor(Xh.dims, [i.to(DEV) for i in Xh.idx], Xh.val.to(DEV), validate=validate)


def factors(dims, R, seed, dtype=torch.float32):
    """(master FP32 host factors, device factors in dtype, host copy of the
    device values widened to FP64)."""
    master = synth.generate_factors(dims, R, seed=seed)
    dev = [u.to(dtype).to(DEV).contiguous() for u in master]
    rounded = [u.to(dtype).to(torch.float64).numpy() for u in master]
    return [u.numpy() for u in master], dev, rounded


def small(name, nnz, dims, seed=None, R=None):
    return synth.WORKLOADS[name].scaled(nnz=nnz, dims=dims, seed=seed, R=R)


def generate(wl, **kw) -> synth.Tensor:
    """``synth.generate`` with the oracle evaluating the planted CP model of
    the planted-value workload (cploss3d)."""
    return synth.generate(wl, model_values=oracle.planted_model, **kw)
