"""Seeded synthetic COO tensors and factor matrices.

These stand in for the paper's real tensors (FROSTT, HaTen2 and CHOA sets of
Table 3 in Sec. 6), which are not available: the same orders (3, 4, 5),
long-tailed mode sizes and power-law slice densities, generated from a seed.
No record of any real dataset is reproduced.

This module is shared by the CUDA path's tests and bench and by the oracle's
tests, so it holds none of the method's arithmetic: it only draws random
coordinates, values and factors.  The planted-model workload's values are the
CP model at the drawn coordinates plus noise; the caller passes the model
evaluator in (``model_values``): the tests pass the oracle's, ``bench.py`` its
own, and this module only adds the noise.

Workloads (the five shapes the build measures and tests on):

  uniform3d_200   200x200x200, 20,000 distinct uniform coordinates, values
                  U(-1,1), FP32 factors N(0,1), R=16.
  zipf3d          1M x 500k x 200k, 100M distinct coordinates, each mode's
                  index Zipf(s=1.1), values lognormal(0,1), R=32.
  zipf4d          50k x 50k x 5k x 1k, 50M coordinates Zipf(s=1.2) per mode
                  (duplicates kept), values U(0,1), R=64.
  cploss3d        200k^3, 20M distinct uniform coordinates, values from a
                  planted rank-16 CP model with N(0,1) factors plus N(0,0.01^2)
                  noise; fitted at R=32.
  zipf5d          8 x 10M x 2M x 100k x 1k, 200M coordinates, mode 0 uniform
                  (the short, heavily contended mode), Zipf(s=1.5) on the
                  others (duplicates kept), values lognormal(0,1), R=16.

Zipf sampling: bounded Zipf over ranks 1..I with p(k) proportional to k^-s,
drawn by inverse CDF (searchsorted on an FP64 CDF); ranks are mapped to
indices through a seeded random permutation of the mode so that hot rows are
not adjacent.  Deduplication (where a workload asks for distinct coordinates)
packs the coordinate into one 64-bit key, takes the distinct keys, tops up
until there are at least nnz of them, then keeps a random nnz-subset.  The
final storage order is random.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, Sequence

import torch


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    dims: tuple[int, ...]
    nnz: int
    index_dist: tuple[str, ...]      # per mode: "uniform" or "zipf"
    zipf_s: float                    # exponent for the "zipf" modes
    distinct: bool                   # deduplicate coordinates
    values: str                      # "uniform_pm1", "uniform01", "lognormal", "planted"
    R: int                           # rank of the fitted factors
    planted_R: int = 0               # rank of the planted model ("planted" values)
    noise_sigma: float = 0.0
    seed: int = 1

    @property
    def order(self) -> int:
        return len(self.dims)

    def scaled(self, nnz: int, dims: Sequence[int] | None = None, name: str | None = None,
               seed: int | None = None, R: int | None = None) -> "Workload":
        """Same distributions, smaller size (for oracle-checkable tests)."""
        return dataclasses.replace(
            self, nnz=int(nnz), dims=tuple(int(d) for d in (dims or self.dims)),
            name=name or f"{self.name}_n{nnz}", seed=self.seed if seed is None else seed,
            R=self.R if R is None else R)


WORKLOADS: dict[str, Workload] = {
    "uniform3d_200": Workload("uniform3d_200", (200, 200, 200), 20_000,
                              ("uniform",) * 3, 0.0, True, "uniform_pm1", 16, seed=1),
    "zipf3d": Workload("zipf3d", (1_000_000, 500_000, 200_000), 100_000_000,
                       ("zipf",) * 3, 1.1, True, "lognormal", 32, seed=2),
    "zipf4d": Workload("zipf4d", (50_000, 50_000, 5_000, 1_000), 50_000_000,
                       ("zipf",) * 4, 1.2, False, "uniform01", 64, seed=3),
    "cploss3d": Workload("cploss3d", (200_000, 200_000, 200_000), 20_000_000,
                         ("uniform",) * 3, 0.0, True, "planted", 32,
                         planted_R=16, noise_sigma=0.01, seed=4),
    "zipf5d": Workload("zipf5d", (8, 10_000_000, 2_000_000, 100_000, 1_000), 200_000_000,
                       ("uniform",) + ("zipf",) * 4, 1.5, False, "lognormal", 16, seed=5),
}


def _gen(device, seed: int) -> torch.Generator:
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return g


def bits_for(dim: int) -> int:
    """Bits needed to hold indices 0..dim-1 (0 for a mode of size 1)."""
    return max(0, int(dim - 1).bit_length())


class _ZipfSampler:
    """Bounded Zipf(s) over ranks 1..dim mapped through a random permutation."""

    def __init__(self, dim: int, s: float, device, g: torch.Generator):
        # the CDF is summed on the host (a sequential FP64 sum), so that the
        # same seed gives the same tensor on any device and in every run
        k = torch.arange(1, dim + 1, dtype=torch.float64)
        cdf = torch.cumsum(k.pow(-float(s)), 0)
        self.cdf = (cdf / cdf[-1]).to(device)
        self.perm = torch.randperm(dim, device=device, generator=g).to(torch.int32)
        self.dim = dim

    def sample(self, n: int, g: torch.Generator) -> torch.Tensor:
        u = torch.rand(n, device=self.cdf.device, dtype=torch.float64, generator=g)
        rank = torch.searchsorted(self.cdf, u).clamp_(max=self.dim - 1)
        return self.perm[rank]


def _draw_coords(wl: Workload, n: int, samplers, g: torch.Generator, device) -> list[torch.Tensor]:
    out = []
    for k, dim in enumerate(wl.dims):
        if wl.index_dist[k] == "zipf":
            out.append(samplers[k].sample(n, g))
        else:
            out.append(torch.randint(0, dim, (n,), device=device, dtype=torch.int32, generator=g))
    return out


def _pack(coords: list[torch.Tensor], dims) -> torch.Tensor:
    key = torch.zeros_like(coords[0], dtype=torch.int64)
    for c, d in zip(coords, dims):
        key = (key << bits_for(d)) | c.to(torch.int64)
    return key


def _unpack(key: torch.Tensor, dims) -> list[torch.Tensor]:
    out = []
    for d in reversed(dims):
        b = bits_for(d)
        out.append((key & ((1 << b) - 1)).to(torch.int32))
        key = key >> b
    return list(reversed(out))


def generate_coords(wl: Workload, device="cpu", seed: int | None = None) -> list[torch.Tensor]:
    """Draw ``wl.nnz`` coordinates (one int32 tensor per mode, random order)."""
    seed = wl.seed if seed is None else seed
    g = _gen(device, seed)
    samplers = [(_ZipfSampler(d, wl.zipf_s, device, g) if wl.index_dist[k] == "zipf" else None)
                for k, d in enumerate(wl.dims)]
    if wl.nnz == 0:
        return [torch.zeros(0, dtype=torch.int32, device=device) for _ in wl.dims]
    if not wl.distinct:
        return _draw_coords(wl, wl.nnz, samplers, g, device)
    total_bits = sum(bits_for(d) for d in wl.dims)
    if total_bits > 63:
        raise ValueError("distinct coordinates need the packed key to fit 63 bits")
    capacity = math.prod(wl.dims)
    if wl.nnz > capacity:
        raise ValueError("more distinct coordinates requested than cells")
    keys = torch.zeros(0, dtype=torch.int64, device=device)
    over = 1.05 if wl.index_dist.count("zipf") == 0 else 1.35
    while keys.numel() < wl.nnz:
        need = wl.nnz - keys.numel()
        batch = int(need * over) + 1024
        fresh = _pack(_draw_coords(wl, batch, samplers, g, device), wl.dims)
        keys = torch.unique(torch.cat([keys, fresh]))
        over *= 1.5
    pick = torch.randperm(keys.numel(), device=device, generator=g)[: wl.nnz]
    return _unpack(keys[pick], wl.dims)


def generate_factors(dims: Sequence[int], R: int, device="cpu", seed: int = 0,
                     dtype=torch.float32) -> list[torch.Tensor]:
    """N(0,1) factor matrices, row-major ``dims[k] x R``."""
    g = _gen(device, seed)
    return [torch.randn((int(d), R), device=device, dtype=torch.float32, generator=g).to(dtype)
            for d in dims]


ModelValues = Callable[[list[torch.Tensor], list[torch.Tensor]], torch.Tensor]


def generate_values(wl: Workload, coords: list[torch.Tensor], device="cpu",
                    seed: int | None = None, model_values: ModelValues | None = None
                    ) -> tuple[torch.Tensor, list[torch.Tensor] | None]:
    """Values for ``coords``.  Returns (values, planted factors or None).

    A "planted" workload needs ``model_values(coords, planted)``: the CP
    model's value at every coordinate (FP64 or FP32, on ``device``)."""
    seed = (wl.seed if seed is None else seed) + 1000
    g = _gen(device, seed)
    n = coords[0].numel()
    if wl.values == "uniform_pm1":
        return torch.rand(n, device=device, generator=g) * 2.0 - 1.0, None
    if wl.values == "uniform01":
        return torch.rand(n, device=device, generator=g), None
    if wl.values == "lognormal":
        return torch.exp(torch.randn(n, device=device, generator=g)), None
    if wl.values == "planted":
        planted = generate_factors(wl.dims, wl.planted_R, device=device, seed=seed + 1)
        if model_values is None:
            raise ValueError(f"workload {wl.name!r} has planted-model values: pass model_values")
        v = model_values(coords, planted).to(device=device, dtype=torch.float64)
        v = (v + wl.noise_sigma * torch.randn(n, device=device, generator=g)).to(torch.float32)
        return v, planted
    raise ValueError(wl.values)


@dataclasses.dataclass
class Tensor:
    """A generated COO tensor (host or device torch tensors)."""
    workload: Workload
    dims: tuple[int, ...]
    idx: list[torch.Tensor]          # int32, one per mode (indices < 2^31)
    val: torch.Tensor                # float32
    planted: list[torch.Tensor] | None = None

    @property
    def nnz(self) -> int:
        return int(self.val.numel())

    def to(self, device) -> "Tensor":
        return Tensor(self.workload, self.dims, [i.to(device) for i in self.idx],
                      self.val.to(device),
                      None if self.planted is None else [p.to(device) for p in self.planted])


def generate(wl: Workload, device="cpu", seed: int | None = None,
             model_values: ModelValues | None = None) -> Tensor:
    coords = generate_coords(wl, device=device, seed=seed)
    val, planted = generate_values(wl, coords, device=device, seed=seed, model_values=model_values)
    return Tensor(wl, tuple(wl.dims), coords, val.to(torch.float32).contiguous(), planted)


def factors_for(wl: Workload, device="cpu", dtype=torch.float32, seed: int | None = None,
                R: int | None = None) -> list[torch.Tensor]:
    """The fitted/input factors of a workload: N(0,1), seed = workload seed + 100."""
    return generate_factors(wl.dims, R or wl.R, device=device,
                            seed=(wl.seed + 100) if seed is None else seed, dtype=dtype)
