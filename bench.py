"""Benchmark: COO MTTKRP throughput (nnz/s, fraction of the HBM roofline) and
CP-loss forward+backward time, FP32 vs BF16 factors, on one GB300 per rank.

Workload (default, the measured shape): zipf3d, a 1M x 500k x 200k COO tensor
with 100M distinct coordinates, each mode's index Zipf(s=1.1), lognormal(0,1)
values, R = 32 FP32 factors (synthetic, seeded; stands in for the paper's
FROSTT-style tensors).

One timed step = one pass of the hot path over the tensor: MTTKRP on every
mode (each on its mode-sorted copy) followed by the CP loss and the gradient
of every factor (pasta_cp_loss_fwd_bwd: one pass per mode over that mode's
sorted copy, the first pass also summing the loss).  The mode sorts are preprocessing: they run
once before timing (the paper treats its sort as given preprocessing and does not time it),
and their time is reported under "preprocess".  `value` = N modes x nnz / (MTTKRP part of the
step), summed over ranks, with device time taken by CUDA events on the
launching stream and the maximum over ranks.  The COO stream (1.6 GB) is
larger than L2, so no L2 flush is inserted.

`--impl reference` times the FP64 CPU oracle on the host cores (a bounded
sample of the same workload); the reference paper has no GPU code.
"""
from __future__ import annotations

import argparse
import gc
import hashlib
import json
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MTTKRP nnz/s & % of HBM roofline; CP-loss fwd+bwd time BF16 vs FP32"
DEFAULT_WORKLOAD = "zipf3d"
LOSS_WORKLOAD = "cploss3d"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="own", choices=["own", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-loss-compare", action="store_true")
    ap.add_argument("--no-als", action="store_true")
    ap.add_argument("--no-tew", action="store_true")
    ap.add_argument("--no-ttm", action="store_true")
    ap.add_argument("--factor-dtype", default="f32", choices=["f32", "bf16", "f16"],
                    help="factor storage type of the timed step (FP32 accumulation either way)")
    ap.add_argument("--nnz", type=float, default=None,
                    help="run the workload's distributions and dims at this many entries "
                         "(small cases for profiling; not a bench line)")
    ap.add_argument("--cpu-sample", type=int, default=12_000_000,
                    help="entries of the workload the CPU oracle runs on")
    ap.add_argument("--no-legs", action="store_true",
                    help="skip the extra measured legs (gather ceiling, L2-flushed MTTKRP, BF16 factors, "
                         "zipf4d and zipf5d)")
    ap.add_argument("--no-multicore", action="store_true",
                    help="skip the multicore CPU baseline (privatized OpenMP MTTKRP)")
    ap.add_argument("--hicoo", action="store_true",
                    help="also time the HiCOO copy's build and MTTKRP against the sorted-copy MTTKRP "
                         "(zipf3d, zipf4d, zipf5d; block sizes 2^7 and 2^8)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload_desc(wl) -> str:
    dims = " x ".join(f"{d:,}" for d in wl.dims)
    what = "distinct" if wl.distinct else "with duplicates"
    dist = "/".join(sorted(set(wl.index_dist)))
    return (f"{wl.name}: {dims}, nnz={wl.nnz:,} {what}, indices {dist}"
            f"{f' s={wl.zipf_s}' if 'zipf' in wl.index_dist else ''}, values {wl.values}, R={wl.R}")


# ------------------------------------------------------------------ clocks --

class ClockSampler:
    """nvidia-smi clock/throttle samples while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            import tempfile
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "20"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            return
        # wait (up to 3 s) for the first sample, so the timed region is covered
        t0 = time.time()
        while time.time() - t0 < 3.0:
            try:
                if os.path.getsize(self.path) > 0:
                    break
            except OSError:
                break
            time.sleep(0.01)

    def stop(self) -> dict | None:
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        sm_sorted = sorted(sm)
        return {"sm_mhz": sm_sorted[len(sm_sorted) // 2] if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------- roofline inputs --

def measured_peak_gbs():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# Kernel groups of the step and the sources their kernels are built from.
KERNEL_SOURCES = {
    "mttkrp": ("stream_kernels.cuh", "stream_launch.cuh", "stream_mttkrp.cu", "mttkrp.cu"),
    "loss_fwd_bwd": ("stream_kernels.cuh", "stream_launch.cuh", "stream_loss_bwd.cu", "cp_loss.cu"),
}
KERNEL_NAMES = {
    "mttkrp": "k_stream<T, N, 0, ...> (MTTKRP)",
    "loss_fwd_bwd": "k_stream<T, N, 2, ...> (loss backward, first pass also sums the loss)",
}


def kernel_source_hash(kernel: str) -> str:
    """Hash of the sources a kernel group is built from (and the shared header)."""
    h = hashlib.sha256()
    for f in (*KERNEL_SOURCES[kernel], "pasta_internal.cuh"):
        with open(os.path.join(ROOT, "paper_1902_03317_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel: str, workload: str):
    """DRAM bytes (read + write) per launch of `kernel` from the committed ncu
    summary profiles/<kernel>_<workload>_traffic.txt, if that capture was taken
    on the current kernel source (else None)."""
    p = os.path.join(ROOT, "profiles", f"{kernel}_{workload}_traffic.txt")
    try:
        kv = {}
        for line in open(p):
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                kv[k.strip()] = v.strip()
        if kv.get("kernel_source_sha256_16") != kernel_source_hash(kernel):
            return None
        return float(kv["dram_bytes_per_launch_mean"])
    except Exception:
        return None


# ------------------------------------------------------------ own (GPU) --

def run_own(args, rank, world, local):
    import torch
    import torch.distributed as dist

    import __graft_entry__
    __graft_entry__.build()
    import paper_1902_03317_gb300 as pasta
    from paper_1902_03317_gb300 import synth

    from paper_1902_03317_gb300 import shard

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1 and not dist.is_initialized():
        # host tensors (timings) over gloo, device tensors (the sharded
        # step's range-end rows and loss) over NCCL
        dist.init_process_group("cpu:gloo,cuda:nccl")

    wl = synth.WORKLOADS[args.workload]
    if args.nnz:
        wl = wl.scaled(nnz=int(args.nnz))
    N = wl.order
    # ---- inputs, resident in HBM
    Xd = synth.generate(wl, device=dev, model_values=planted_model_values)
    fdt = {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16}[args.factor_dtype]
    Us = [u.to(fdt).contiguous() for u in synth.factors_for(wl, device=dev)]
    X = pasta.CooTensor(Xd.dims, Xd.idx, Xd.val)
    # rows of each factor touched (algorithmic bytes), counted before timing
    touched = [int(torch.unique(ix).numel()) for ix in Xd.idx]
    t_sort = timed_sorts(X, N)
    Ms = [torch.empty((wl.dims[n], wl.R), device=dev) for n in range(N)]
    stream = torch.cuda.current_stream()
    # With several ranks the tensor is split, not replicated: rank r takes
    # positions [lo, hi) of every sorted copy (shard.step_range), computes
    # its partial MTTKRPs and its partial loss and gradients with the range
    # calls, and the rows cut by range ends are completed across ranks
    # (shard.complete_boundary_rows; the loss by an all-reduce).  Each rank
    # then holds the complete rows its range reaches.
    sharded = world > 1
    lo, hi = shard.step_range(wl.nnz, world, rank) if sharded else (0, wl.nnz)
    shared_rows = []  # per mode: rows this rank's range may share with other ranks
    if sharded:
        for n in range(N):
            sidx = X.copy_out(n)[0][n]
            first, last = (int(sidx[lo]), int(sidx[hi - 1])) if hi > lo else (-1, -1)
            del sidx
            shared_rows.append(shard.boundary_rows(first, last, dev))

    def step(ev=None):
        # ev: 2N + 2 events: [mttkrp n start, end]*N, loss fwd+bwd start/end
        for n in range(N):
            if ev is not None:
                ev[2 * n].record(stream)
            if sharded:
                pasta.mttkrp_range(X, Us, n, lo, hi, out=Ms[n])
                shard.sum_rows(Ms[n], shared_rows[n])
            else:
                pasta.mttkrp(X, Us, n, out=Ms[n])
            if ev is not None:
                ev[2 * n + 1].record(stream)
        if ev is not None:
            ev[2 * N].record(stream)
        if sharded:
            loss, G = pasta.cp_loss_fwd_bwd_range(X, Us, lo, hi)
            dist.all_reduce(loss.reshape(1))
            for n in range(N):
                shard.sum_rows(G[n], shared_rows[n])
        else:
            pasta.cp_loss_fwd_bwd(X, Us)
        if ev is not None:
            ev[2 * N + 1].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(2 * N + 2)] for _ in range(args.steps)]
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    clocks.start()
    torch.cuda.synchronize()
    start.record(stream)
    for k in range(args.steps):
        step(evs[k])
    end.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    total_ms = start.elapsed_time(end)
    K = args.steps
    per_mode_ms = [sum(evs[k][2 * n].elapsed_time(evs[k][2 * n + 1]) for k in range(K)) / K for n in range(N)]
    loss_ms = sum(evs[k][2 * N].elapsed_time(evs[k][2 * N + 1]) for k in range(K)) / K
    sweep_ms = sum(per_mode_ms)
    step_ms = total_ms / K
    if world > 1:
        t = torch.tensor([sweep_ms, step_ms], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        sweep_ms, step_ms = float(t[0]), float(t[1])

    nnz = wl.nnz
    # sharded: the ranks split one tensor (strong scaling); one rank: the whole
    value = N * nnz / (sweep_ms * 1e-3)
    # Algorithmic (compulsory) bytes, factor element size s: each pass over the
    # COO stream reads N 32-bit indices and one FP32 value per entry; every
    # factor row the pass needs is read once; each output row written once.
    es = Us[0].element_size()
    coo = nnz * (4 * N + 4)
    rows = [touched[k] * wl.R * es for k in range(N)]
    out = [wl.dims[n] * wl.R * 4 for n in range(N)]
    alg = {
        "mttkrp": ([coo + sum(rows) - rows[n] + out[n] for n in range(N)], sweep_ms, N),
        "loss_fwd_bwd": ([coo + sum(rows) + out[n] for n in range(N)], loss_ms, N),
    }
    peak, peak_src = measured_peak_gbs()
    rooflines = {}
    for kname, (bytes_per_launch, ms, launches) in alg.items():
        achieved = sum(bytes_per_launch) / (ms * 1e-3) / 1e9
        rooflines[kname] = {
            "bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4),
            "traffic": profiled_traffic(kname, args.workload) if args.factor_dtype == "f32" else None,
            "kernel": KERNEL_NAMES[kname], "group": kname, "launches_per_step": launches,
            "ms_per_step": round(ms, 4),
            "alg_bytes_per_launch": bytes_per_launch,
            "peak_source": f"{peak_src} hbm_gbs (MEASURED_PEAKS.json)",
            "frac_vs_8TBs": round(achieved / 8000.0, 4)}
    dominant = max(rooflines, key=lambda k: rooflines[k]["ms_per_step"])

    result = {
        "metric": METRIC, "value": value, "unit": "nnz/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True,
        "scaling": "strong", "vs_baseline": None, "dtype": args.factor_dtype, "data": "synthetic",
        "config": {"workload": workload_desc(wl), "step": "MTTKRP every mode + CP loss and all gradients (one pass per mode over its sorted copy, the first also summing the loss)",
                   "l2": "no flush: inputs larger than L2 (COO stream 1.6 GB)",
                   "parallelism": (f"entries split over {world} GPUs (positions [lo, hi) of every sorted copy "
                                   f"per rank; range-end rows and the loss summed over NCCL)") if world > 1
                   else "single GPU"},
        "roofline": rooflines[dominant],
        "rooflines": rooflines,
        "breakdown_ms": {"mttkrp_per_mode": [round(x, 4) for x in per_mode_ms],
                         "loss_fwd_bwd": round(loss_ms, 4)},
        "preprocess": sort_roofline(t_sort, nnz, N, peak),
        "gpu_launches": args.steps * (N + N + 1),
        "clocks": clk,
    }
    del Xd
    torch.cuda.empty_cache()

    if not args.no_legs and rank == 0:
        result["gather_ceiling"] = gather_ceiling(pasta, X, Us, wl, per_mode_ms, peak, args)
        result["l2_flush"] = l2_flush_leg(pasta, X, Us, wl, per_mode_ms, args)
        if args.factor_dtype == "f32":
            result["bf16_factors"] = bf16_leg(pasta, X, wl, touched, peak, args, dev)
    if not args.no_ttm and rank == 0:
        result["ttm_ttv"] = ttm_timing(pasta, X, wl, peak, args)
    if not args.no_tew and rank == 0:
        result["tew_ts"] = tew_ts_timing(pasta, X, N, nnz, peak, args)
    if not args.no_als and rank == 0 and args.factor_dtype == "f32":
        result["cp_als"] = als_timing(pasta, X, Us, wl, args, sweep_ms)
    if not args.no_loss_compare and rank == 0:
        result["cp_loss"] = loss_compare(pasta, synth, dev, args)
    if not args.no_e2e:
        result["e2e"] = e2e(pasta, synth, wl, dev, args, world)
    if rank == 0 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline(wl, args, pasta, dev)
    X.close()
    del Us, Ms
    torch.cuda.empty_cache()
    if rank == 0 and not args.no_multicore and not args.no_cpu_baseline and not args.nnz:
        result["cpu_multicore"] = cpu_multicore(wl, args)
    if args.hicoo and rank == 0:
        result["hicoo"] = {name: hicoo_leg(pasta, synth, name, args, dev) for name in ("zipf3d", "zipf4d", "zipf5d")}
    if not args.no_legs and rank == 0 and not args.nnz:
        result["workloads"] = {name: workload_leg(pasta, synth, name, dts, peak, args, dev, loss)
                               for name, dts, loss in (("zipf4d", ("f32", "bf16"), False),
                                                       ("zipf5d", ("bf16",), True))}
    if rank == 0:
        print(json.dumps(result), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def _time_ms(fn, reps):
    """Mean device time of fn() over reps calls (CUDA events on the current stream)."""
    import torch
    fn()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def mttkrp_alg_bytes(nnz, N, R, es, touched, dims, n):
    """Compulsory bytes of one mode-n MTTKRP: the COO stream (N 32-bit
    indices + FP32 value per entry), every touched row of the other factors
    (element size es) once, the FP32 output once."""
    return nnz * (4 * N + 4) + sum(touched[k] * R * es for k in range(N) if k != n) + dims[n] * R * 4


def gather_ceiling(pasta, X, Us, wl, mttkrp_ms, peak, args):
    """pasta_gather_probe per mode: the same kernel, launch and row gathers as
    the MTTKRP with no arithmetic into output rows.  Its time is the ceiling
    the MTTKRP kernel can reach with these gathers; also reported as the
    gathered bytes per second through L1/L2 (every entry's N-1 rows of R
    elements, hits included)."""
    import torch
    N = wl.order
    sink = torch.empty(1 << 22, dtype=torch.float32, device=X.device)
    K = max(5, args.steps // 2)
    es = Us[0].element_size()
    out = {"what": "pasta_gather_probe: MTTKRP's staging, batches and row gathers, no arithmetic or output rows",
           "ms_per_mode": [], "gathered_bytes_per_mode": wl.nnz * (N - 1) * wl.R * es,
           "gathered_gbs": [], "mttkrp_ms_per_mode": [round(x, 4) for x in mttkrp_ms],
           "mttkrp_over_probe": []}
    for n in range(N):
        ms = _time_ms(lambda: pasta.gather_probe(X, Us, n, sink=sink), K)
        out["ms_per_mode"].append(round(ms, 4))
        out["gathered_gbs"].append(round(out["gathered_bytes_per_mode"] / (ms * 1e-3) / 1e9, 1))
        out["mttkrp_over_probe"].append(round(mttkrp_ms[n] / ms, 3))
    return out


def l2_flush_leg(pasta, X, Us, wl, mttkrp_ms, args):
    """MTTKRP per mode with L2 flushed before every call (a 512 MB buffer
    written between calls, outside the timed events), against the unflushed
    back-to-back calls of the timed step: what carrying factor rows in L2
    from one call to the next (evict-last policy) is worth."""
    import torch
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=X.device)
    K = max(5, args.steps // 2)
    Ms = [torch.empty((wl.dims[n], wl.R), device=X.device) for n in range(wl.order)]
    flushed = []
    for n in range(wl.order):
        tot = 0.0
        for _ in range(K):
            flush.fill_(1)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            pasta.mttkrp(X, Us, n, out=Ms[n])
            b.record()
            torch.cuda.synchronize()
            tot += a.elapsed_time(b)
        flushed.append(round(tot / K, 4))
    return {"flush": "512 MB written before each call (L2 is 126 MB)", "flushed_ms_per_mode": flushed,
            "unflushed_ms_per_mode": [round(x, 4) for x in mttkrp_ms],
            "flushed_over_unflushed": [round(f / u, 3) for f, u in zip(flushed, mttkrp_ms)]}


def bf16_leg(pasta, X, wl, touched, peak, args, dev):
    """The benchmark tensor with BF16 factors (FP32 accumulation): MTTKRP per
    mode and the fused loss + gradients, with the compulsory-byte rooflines."""
    import torch
    from paper_1902_03317_gb300 import synth
    N = wl.order
    Ub = [u.to(torch.bfloat16).contiguous() for u in synth.factors_for(wl, device=dev)]
    K = max(5, args.steps // 2)
    ms = [_time_ms(lambda: pasta.mttkrp(X, Ub, n), K) for n in range(N)]
    sink = torch.empty(1 << 22, dtype=torch.float32, device=dev)
    probe = [_time_ms(lambda: pasta.gather_probe(X, Ub, n, sink=sink), K) for n in range(N)]
    loss_ms = _time_ms(lambda: pasta.cp_loss_fwd_bwd(X, Ub), K)
    alg = [mttkrp_alg_bytes(wl.nnz, N, wl.R, 2, touched, wl.dims, n) for n in range(N)]
    gbs = sum(alg) / (sum(ms) * 1e-3) / 1e9
    lalg = [wl.nnz * (4 * N + 4) + sum(touched[k] * wl.R * 2 for k in range(N)) + wl.dims[n] * wl.R * 4
            for n in range(N)]
    lgbs = sum(lalg) / (loss_ms * 1e-3) / 1e9
    return {"mttkrp_ms_per_mode": [round(x, 4) for x in ms], "value_nnz_per_s": N * wl.nnz / (sum(ms) * 1e-3),
            "gather_probe_ms_per_mode": [round(x, 4) for x in probe],
            "mttkrp_over_probe": [round(a / b, 3) for a, b in zip(ms, probe)],
            "mttkrp_alg_bytes_per_mode": alg, "mttkrp_achieved_gbs": round(gbs, 1),
            "mttkrp_frac": round(gbs / peak, 4), "loss_fwd_bwd_ms": round(loss_ms, 4),
            "loss_achieved_gbs": round(lgbs, 1), "loss_frac": round(lgbs / peak, 4)}


def workload_leg(pasta, synth, name, dts, peak, args, dev, with_loss):
    """Another configuration at its full size: generate, sort every mode,
    then MTTKRP per mode (and, with_loss, the fused loss + gradients) for each
    factor type, with compulsory-byte rooflines.  Parity of these shapes
    against the oracle is covered by the test suite (full-size sampled-row
    checks, scaled element-wise checks)."""
    import torch
    wl = synth.WORKLOADS[name]
    N = wl.order
    Xd = synth.generate(wl, device=dev, model_values=planted_model_values)
    touched = [int(torch.unique(ix).numel()) for ix in Xd.idx]
    X = pasta.CooTensor(Xd.dims, Xd.idx, Xd.val)
    del Xd
    torch.cuda.empty_cache()
    t_sort = [round(x, 3) for x in timed_sorts(X, N)]
    out = {"workload": workload_desc(wl), "sort_ms_per_mode": t_sort}
    K = max(5, args.steps // 3)
    for dt in dts:
        tdt = {"f32": torch.float32, "bf16": torch.bfloat16}[dt]
        es = 4 if dt == "f32" else 2
        Us = [u.to(tdt).contiguous() for u in synth.factors_for(wl, device=dev)]
        Ms = [torch.empty((wl.dims[n], wl.R), device=dev) for n in range(N)]
        ms = [_time_ms(lambda: pasta.mttkrp(X, Us, n, out=Ms[n]), K) for n in range(N)]
        alg = [mttkrp_alg_bytes(wl.nnz, N, wl.R, es, touched, wl.dims, n) for n in range(N)]
        gbs = sum(alg) / (sum(ms) * 1e-3) / 1e9
        leg = {"mttkrp_ms_per_mode": [round(x, 4) for x in ms],
               "value_nnz_per_s": N * wl.nnz / (sum(ms) * 1e-3),
               "mttkrp_alg_bytes_per_mode": alg, "mttkrp_achieved_gbs": round(gbs, 1),
               "mttkrp_frac": round(gbs / peak, 4)}
        if with_loss:
            lms = _time_ms(lambda: pasta.cp_loss_fwd_bwd(X, Us), K)
            lalg = sum(wl.nnz * (4 * N + 4) + sum(touched[k] * wl.R * es for k in range(N)) + wl.dims[n] * wl.R * 4
                       for n in range(N))
            leg["loss_fwd_bwd_ms"] = round(lms, 4)
            leg["loss_achieved_gbs"] = round(lalg / (lms * 1e-3) / 1e9, 1)
            leg["loss_frac"] = round(lalg / (lms * 1e-3) / 1e9 / peak, 4)
        out[dt] = leg
        del Us, Ms
    X.close()
    torch.cuda.empty_cache()
    return out


def hicoo_leg(pasta, synth, name, args, dev):
    """HiCOO (row f3): build time, block count and MTTKRP per mode from the
    HiCOO copy, next to the sorted-copy MTTKRP on the same tensor and FP32
    factors, with the relative difference of their outputs."""
    import torch
    wl = synth.WORKLOADS[name]
    if args.nnz:
        wl = wl.scaled(nnz=int(args.nnz))
    Xd = synth.generate(wl, device=dev, model_values=planted_model_values)
    Us = [u.contiguous() for u in synth.factors_for(wl, device=dev)]
    X = pasta.CooTensor(Xd.dims, Xd.idx, Xd.val)
    del Xd
    X.sort_all()
    out = {"workload": workload_desc(wl)}
    K = max(3, args.steps // 6)
    for bits in (7, 8):
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        nb = pasta.hicoo(X, bits)
        b.record()
        torch.cuda.synchronize()
        res = {"nblocks": nb, "build_ms": round(a.elapsed_time(b), 2), "sorted_ms_per_mode": [],
               "hicoo_ms_per_mode": [], "rel_diff_per_mode": []}
        for n in range(wl.order):
            M = pasta.mttkrp(X, Us, n)
            H = pasta.hicoo_mttkrp(X, Us, n)
            res["rel_diff_per_mode"].append(float((H.double() - M.double()).norm() / M.double().norm()))
            res["sorted_ms_per_mode"].append(round(_time_ms(lambda: pasta.mttkrp(X, Us, n, out=M), K), 4))
            res["hicoo_ms_per_mode"].append(round(_time_ms(lambda: pasta.hicoo_mttkrp(X, Us, n, out=H), K), 4))
            del M, H
        out[f"b{bits}"] = res
    X.close()
    del Us
    torch.cuda.empty_cache()
    return out


def timed_sorts(X, N):
    """Sort every mode in the order sort_all uses (0, N-1, ..., 1: each copy
    after the first re-sorted from the next mode's copy on its own field),
    each timed with CUDA events; returns ms indexed by mode."""
    import torch
    t = [0.0] * N
    for n in [0] + list(range(N - 1, 0, -1)):
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        X.sort_by_mode(n)
        e1.record()
        torch.cuda.synchronize()
        t[n] = e0.elapsed_time(e1)
    return t


def sort_roofline(t_sort, nnz, N, peak):
    """Mode sorts (preprocessing, timed once per mode with CUDA events; the
    first includes growing the handle's scratch buffer).  Compulsory bytes per
    mode: read the creation-order copy (N indices + value) and write the
    sorted copy (N indices + value); the permutation is built only when asked
    for."""
    alg = nnz * (8 * N + 8)
    ms = sum(t_sort) / len(t_sort)
    achieved = alg / (ms * 1e-3) / 1e9
    return {"sort_ms_per_mode": [round(x, 2) for x in t_sort], "alg_bytes_per_mode": alg,
            "achieved_gbs": round(achieved, 1), "frac": round(achieved / peak, 4),
            "note": ("LSD radix passes of up to 9-bit digits over (64-bit key, 32-bit value) pairs, 24 bytes "
                     "per entry per pass; mode 0 from the creation-order copy, then modes N-1, ..., 1, each "
                     "from the next mode's copy on its own index field only")}


def als_timing(pasta, X, Us, wl, args, mttkrp_ms):
    """CP-ALS sweeps (pasta_cp_als_sweep) on the benchmark tensor from the
    benchmark's factors: one warm-up sweep, then K timed with CUDA events
    (each sweep ends with one stream synchronisation for its status); then K
    sweeps through the driver (pasta_cp_als) from where those ended (the
    driver's init clone is inside its timed region)."""
    import torch
    U = [u.clone() for u in Us]
    pasta.cp_als_sweep(X, U)
    K = max(3, args.steps // 2)
    fits = []
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(K):
        _, fit = pasta.cp_als_sweep(X, U)
        fits.append(fit)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / K
    # the same K sweeps through the driver (pasta_cp_als), which keeps each
    # factor's Gram matrix between sweeps
    U0 = [u.clone() for u in U]
    torch.cuda.synchronize()
    e0.record()
    _, _, dfits = pasta.cp_als(X, wl.R, max_sweeps=K, tol=-1.0, init=U0)
    e1.record()
    torch.cuda.synchronize()
    ms_drv = e0.elapsed_time(e1) / K
    return {"workload": f"{wl.name}, R={wl.R} FP32, factors from the benchmark start",
            "sweeps_timed": K, "ms_per_sweep": round(ms, 4),
            "driver_ms_per_sweep": round(ms_drv, 4),
            "mttkrp_ms_per_sweep": round(mttkrp_ms, 4),
            "other_ms_per_sweep": round(ms - mttkrp_ms, 4),
            "fit_after_each": [round(float(f), 6) for f in fits]}


def tew_ts_timing(pasta, X, N, nnz, peak, args):
    """TS (Z = X * s) and TEW-eq (Z = X + Y) on the benchmark tensor into a
    reused output handle, K calls each timed with CUDA events.  Compulsory
    bytes per entry: TS reads X's N indices and value and writes Z's (8N + 8);
    TEW-eq also reads Y's value and, to check the shared coordinates, Y's N
    indices (12N + 12).  TEW-eq synchronises once per call (the check)."""
    import torch
    Y = pasta.ts(X, "mul", 0.5)
    Z = pasta.ts(X, "add", 1.0)
    out = {}
    K = max(3, args.steps // 3)
    for name, call, per_entry in (("ts_mul", lambda: pasta.ts(X, "mul", 1.5, out=Z), 8 * N + 8),
                                  ("tew_eq_add", lambda: pasta.tew_eq(X, Y, "add", out=Z), 12 * N + 12)):
        call()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(K):
            call()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / K
        gbs = per_entry * nnz / (ms * 1e-3) / 1e9
        out[name] = {"ms_per_call": round(ms, 4), "alg_bytes_per_call": per_entry * nnz,
                     "achieved_gbs": round(gbs, 1), "frac": round(gbs / peak, 4), "calls_timed": K}
    Y.close()
    Z.close()
    return out


def ttm_timing(pasta, X, wl, peak, args):
    """Mode-n fiber tables (preprocessing, timed once) and TTM (R = 32, FP32)
    / TTV on the benchmark tensor, every mode, CUDA events.  Compulsory bytes
    of one TTM: the view's stream (fiber id, i_n and value: 12 B per entry),
    U's touched rows and the nfibs x R output; TTV the same with R = 1."""
    import torch
    out = {}
    K = max(3, args.steps // 3)
    for n in range(wl.order):
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        nf = pasta.fibers(X, n)
        e1.record()
        torch.cuda.synchronize()
        fib_ms = e0.elapsed_time(e1)
        U = torch.randn(wl.dims[n], 32, device=X.device)
        v = torch.randn(wl.dims[n], device=X.device)
        rows = min(wl.dims[n], wl.nnz)  # upper bound on touched rows
        res = {"nfibs": nf, "fiber_table_ms": round(fib_ms, 3)}
        for name, call, R in (("ttm_r32", lambda: pasta.ttm(X, U, n), 32), ("ttv", lambda: pasta.ttv(X, v, n), 1)):
            call()
            torch.cuda.synchronize()
            e0.record()
            for _ in range(K):
                call()
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / K
            alg = wl.nnz * 12 + rows * R * 4 + nf * R * 4
            gbs = alg / (ms * 1e-3) / 1e9
            res[name] = {"ms": round(ms, 4), "alg_bytes": alg, "achieved_gbs": round(gbs, 1),
                         "frac": round(gbs / peak, 4)}
        out[f"mode{n}"] = res
    return out


def planted_model_values(coords, planted):
    """Values of the planted-model workload before noise: the CP model
    sum_r prod_k A_k(i_k, r) at every coordinate, FP64, in chunks on the
    coordinates' device (input preparation; the tests make the same values
    with the oracle's evaluator)."""
    import torch
    dev = coords[0].device
    n = coords[0].numel()
    A64 = [A.to(device=dev, dtype=torch.float64) for A in planted]
    out = torch.empty(n, dtype=torch.float64, device=dev)
    step = 1 << 22
    for lo in range(0, n, step):
        acc = None
        for c, A in zip(coords, A64):
            rows = A[c[lo:lo + step].long()]
            acc = rows if acc is None else acc * rows
        out[lo:lo + step] = acc.sum(dim=1)
    return out


def loss_compare(pasta, synth, dev, args):
    """CP-loss forward+backward time, FP32 vs BF16 factors (cploss3d)."""
    import torch
    wl = synth.WORKLOADS[LOSS_WORKLOAD]
    Xd = synth.generate(wl, device=dev, model_values=planted_model_values)
    X = pasta.CooTensor(Xd.dims, Xd.idx, Xd.val)
    X.sort_by_mode(0)
    del Xd
    X.sort_all()
    out = {"workload": workload_desc(wl), "path": "autograd CPLoss, forward over the mode-0 copy"}
    stream = torch.cuda.current_stream()
    for bwd, tag in ((-2, "per_mode"), (0, "one_pass")):
        for name, dt in (("fp32", torch.float32), ("bf16", torch.bfloat16)):
            Us = [u.requires_grad_(True) for u in synth.factors_for(wl, device=dev, dtype=dt)]
            for _ in range(3):
                pasta.cp_loss(X, Us, bwd).backward()
            reps = max(5, args.steps)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record(stream)
            for _ in range(reps):
                for u in Us:
                    u.grad = None
                pasta.cp_loss(X, Us, bwd).backward()
            b.record(stream)
            torch.cuda.synchronize()
            out[f"{name}_fwd_bwd_ms_{tag}"] = round(a.elapsed_time(b) / reps, 4)
    best = {n: min(out[f"{n}_fwd_bwd_ms_per_mode"], out[f"{n}_fwd_bwd_ms_one_pass"]) for n in ("fp32", "bf16")}
    out["fp32_fwd_bwd_ms"] = best["fp32"]
    out["bf16_fwd_bwd_ms"] = best["bf16"]
    out["bf16_speedup"] = round(best["fp32"] / best["bf16"], 3)
    X.close()
    torch.cuda.empty_cache()
    return out


def e2e(pasta, synth, wl, dev, args, world):
    """Same metric through the public API from pinned host buffers: every step
    copies the COO tensor and factors in, builds the handle and sorted
    copies, runs the MTTKRP sweep and reads every output back."""
    import torch
    Xh = synth.generate(wl, device=dev, model_values=planted_model_values)
    idx_h = [i.cpu().pin_memory() for i in Xh.idx]
    val_h = Xh.val.cpu().pin_memory()
    Uh = [u.cpu().pin_memory() for u in synth.factors_for(wl, device=dev)]
    del Xh
    torch.cuda.empty_cache()
    N = wl.order
    outs = [torch.empty((wl.dims[n], wl.R), dtype=torch.float32).pin_memory() for n in range(N)]
    h2d = sum(t.numel() * t.element_size() for t in idx_h + [val_h] + Uh)
    d2h = sum(t.numel() * t.element_size() for t in outs)

    # Streams: `side` carries the factor upload (overlapping the create and
    # the first sort) and each output's download (overlapping later work);
    # `aux` sorts modes 1..N-1 (each derived from the previous mode's copy)
    # while the main stream runs the MTTKRPs of the modes already sorted.
    # Sorts share the handle's scratch buffer, so they stay on one stream;
    # MTTKRP n waits for sort n's event.
    side = torch.cuda.Stream(device=dev)
    aux = torch.cuda.Stream(device=dev)
    main = torch.cuda.current_stream(dev)

    def one(marks=None):
        # the COO arrays go from pinned host memory straight into the
        # handle's creation-order copy; the factors follow on the side stream
        # (marks: events recorded on the main stream after the create with
        # its copy and after the first sort, for the per-step phase times)
        # (create and the mode-0 sort in one call: the second half of the COO
        # is copied in while the first half sorts)
        X = pasta.CooTensor(wl.dims, idx_h, val_h, validate=False, device=dev, sort_mode=0)
        if marks is not None:
            marks[0].record()
        side.wait_stream(main)
        with torch.cuda.stream(side):
            Us = [pasta.copy_(torch.empty(u.shape, dtype=u.dtype, device=dev), u) for u in Uh]
        if marks is not None:
            marks[1].record()
        aux.wait_stream(main)
        sorted_ev = [None]
        with torch.cuda.stream(aux):
            for n in range(N - 1, 0, -1):  # each from the next mode's copy (see sort_all)
                X.sort_by_mode(n)
                sorted_ev.append(aux.record_event())
        main.wait_stream(side)
        for u in Us:
            u.record_stream(main)
        order = [0] + list(range(N - 1, 0, -1))  # modes in the order their copies appear
        for i, n in enumerate(order):
            if sorted_ev[i] is not None:
                main.wait_event(sorted_ev[i])
            M = pasta.mttkrp(X, Us, n)
            side.wait_stream(main)
            with torch.cuda.stream(side):
                pasta.copy_(outs[n], M)
            M.record_stream(side)
        torch.cuda.synchronize()
        X.close()

    for _ in range(3):  # untimed: the first steps after pinning the host buffers ran slow copies
        one()
    # one instrumented step (host clock, synchronised between phases)
    br = {}

    def mark(name, t_prev):
        torch.cuda.synchronize()
        t = time.perf_counter()
        br[name] = round((t - t_prev) * 1e3, 2)
        return t

    t = time.perf_counter()
    X = pasta.CooTensor(wl.dims, idx_h, val_h, validate=False, device=dev)
    t = mark("create_with_coo_h2d", t)
    Us = [pasta.copy_(torch.empty(u.shape, dtype=u.dtype, device=dev), u) for u in Uh]
    t = mark("factors_h2d", t)
    X.sort_all()
    t = mark("sort_all_modes", t)
    Ms = [pasta.mttkrp(X, Us, n) for n in range(N)]
    t = mark("mttkrp_all_modes", t)
    for n in range(N):
        pasta.copy_(outs[n], Ms[n])
    t = mark("d2h", t)
    X.close()
    del Ms, Us
    mark("destroy", t)
    steps = max(2, min(args.steps, 20))
    torch.cuda.synchronize()
    # host-timed steps: Python's cyclic garbage collector is paused while
    # they run, as timeit does
    gc.collect()
    gc_was_on = gc.isenabled()
    gc.disable()
    # per step: host time, the main stream's device time (events), and the
    # caching allocator's device allocations (to tell host stalls, device
    # stalls and cudaMalloc calls apart)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    mk = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    n_alloc = []
    total = 0.0
    per_step = []
    for k in range(steps):
        a0 = torch.cuda.memory_stats(dev).get("num_device_alloc", 0)
        ts = time.perf_counter()
        ev[k][0].record()
        one(mk[k])  # ends with a device synchronisation
        ev[k][1].record()
        te = time.perf_counter() - ts
        total += te
        per_step.append(round(te * 1e3, 2))
        n_alloc.append(torch.cuda.memory_stats(dev).get("num_device_alloc", 0) - a0)
    torch.cuda.synchronize()
    dt = total / steps
    if gc_was_on:
        gc.enable()
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([dt], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dt = float(t[0])
    torch.cuda.empty_cache()
    return {"value": world * N * wl.nnz / dt, "unit": "nnz/s", "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "ms_per_step": dt * 1e3, "steps": steps,
            "median_step_ms": sorted(per_step)[len(per_step) // 2],
            "includes": ("create from pinned host COO with the mode-0 sort (pasta_coo_create_sorted: the second "
                         "half copied in while the first half sorts, then a merge), H2D of factors, sorts of the "
                         "other modes, MTTKRP every mode, D2H of outputs (factor upload and output downloads on a "
                         "side stream; sorts of modes N-1..1 on a second stream, overlapping the MTTKRPs of the "
                         "modes sorted before); every host<->device copy through the library (SM-driven copies "
                         "of pinned host memory)"),
            "breakdown_ms": br, "per_step_ms": per_step,
            "per_step_device_ms": [round(a.elapsed_time(b), 2) for a, b in ev],
            "per_step_phases_ms": [[round(e0.elapsed_time(m0), 2), round(m0.elapsed_time(m1), 2),
                                    round(m1.elapsed_time(e1), 2)] for (e0, e1), (m0, m1) in zip(ev, mk)],
            "phases": ("create with the COO H2D and the mode-0 sort (overlapped); the factor upload's issue; "
                       "the rest (later sorts, MTTKRPs, downloads)"),
            "per_step_device_allocs": n_alloc}


# ----------------------------------------------------------- CPU oracle --

def oracle_sample(wl, sample: int):
    """A bounded, seeded sample of the workload for the CPU oracle: the first
    `sample` entries of the generated tensor (its storage order is random)."""
    import numpy as np
    import torch
    from paper_1902_03317_gb300 import synth
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    Xd = synth.generate(wl, device=dev, model_values=planted_model_values)
    n = min(sample, wl.nnz)
    idx = [i[:n].cpu().numpy().astype(np.uint32) for i in Xd.idx]
    val = Xd.val[:n].cpu().numpy().astype(np.float64)
    del Xd
    U = [u.double().numpy() for u in synth.factors_for(wl)]
    return idx, val, U, n


def cpu_baseline(wl, args, pasta=None, dev=None):
    """The FP64 oracle, one thread, on a bounded sample of the workload (all
    modes).  The same sample also runs through the library on the GPU, and
    the relative Frobenius error of each mode's output against the oracle's
    is reported."""
    import numpy as np
    import oracle
    idx, val, U, n = oracle_sample(wl, args.cpu_sample)
    t0 = time.perf_counter()
    refs = [oracle.mttkrp(wl.dims, idx, val, U, mode, wl.R) for mode in range(wl.order)]
    dt = time.perf_counter() - t0
    out = {"value": wl.order * n / dt, "unit": "nnz/s", "cores": 1, "kind": "oracle",
           "sample": f"first {n:,} of {wl.nnz:,} entries (random storage order), MTTKRP on all "
                     f"{wl.order} modes, FP64 C oracle, 1 thread: {dt:.1f} s"}
    if pasta is not None:
        import torch
        Xs = pasta.CooTensor(wl.dims, [torch.from_numpy(i.astype(np.int32)).to(dev) for i in idx],
                             torch.from_numpy(val.astype(np.float32)).to(dev))
        Ug = [torch.from_numpy(u.astype(np.float32)).to(dev) for u in U]
        errs = []
        for mode in range(wl.order):
            M = pasta.mttkrp(Xs, Ug, mode).double().cpu().numpy()
            errs.append(float(np.linalg.norm(M - refs[mode]) / np.linalg.norm(refs[mode])))
        Xs.close()
        out["gpu_rel_err_vs_oracle"] = errs
    return out


def cpu_multicore(wl, args):
    """The paper's multicore MTTKRP (Sec. 5.3: parallel loop over the stored
    entries, privatized outputs, then a parallel reduction), FP32, on every
    host core, over the whole workload, all modes.  A baseline only."""
    import numpy as np
    import oracle
    from paper_1902_03317_gb300 import synth
    import torch
    Xd = synth.generate(wl, device="cuda" if torch.cuda.is_available() else "cpu",
                        model_values=planted_model_values)
    idx = [i.cpu().numpy().astype(np.uint32) for i in Xd.idx]
    val = Xd.val.cpu().numpy()
    del Xd
    U = [u.numpy() for u in synth.factors_for(wl)]
    threads = oracle.cpu_threads()
    oracle.mttkrp_privatized(wl.dims, [i[:100_000] for i in idx], val[:100_000], U, 0)  # warm-up
    times = []
    for mode in range(wl.order):
        t0 = time.perf_counter()
        oracle.mttkrp_privatized(wl.dims, idx, val, U, mode)
        times.append(time.perf_counter() - t0)
    dt = sum(times)
    return {"value": wl.order * wl.nnz / dt, "unit": "nnz/s", "cores": threads,
            "kind": "privatized OpenMP MTTKRP, FP32 (the paper's Sec. 5.3 scheme)",
            "s_per_mode": [round(t, 3) for t in times], "nproc": os.cpu_count(),
            "sample": f"whole workload ({wl.nnz:,} entries), all {wl.order} modes"}


def run_reference(args, rank, world):
    if rank != 0:
        return
    from paper_1902_03317_gb300 import synth
    import oracle
    oracle.build()
    wl = synth.WORKLOADS[args.workload]
    sample = max(100_000, args.cpu_sample // max(1, args.steps))
    idx, val, U, n = oracle_sample(wl, sample)
    for _ in range(args.warmup):
        oracle.mttkrp(wl.dims, idx, val, U, 0, wl.R)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for mode in range(wl.order):
            oracle.mttkrp(wl.dims, idx, val, U, mode, wl.R)
    dt = (time.perf_counter() - t0) / args.steps
    value = wl.order * n / dt
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "nnz/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_desc(wl), "step": f"oracle MTTKRP on all modes over {n:,} sampled entries"},
        "cpu_baseline": {"value": value, "unit": "nnz/s", "cores": 1, "kind": "oracle",
                         "sample": f"first {n:,} of {wl.nnz:,} entries per step"},
        "e2e": {"value": value, "unit": "nnz/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    run_own(args, rank, world, local)


if __name__ == "__main__":
    main()
