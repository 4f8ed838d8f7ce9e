#!/usr/bin/env python3
"""Throughput benchmark of the signature-kernel Gram path on GB300.

Workload ("gram128"): X and Y are 128 Brownian paths each on [0, 1], 257 points, d = 8,
increments N(0, 1/256) per coordinate (seeds 3 and 4; other ranks use their own seeds), solved
with the polynomial approximation scheme of order 6 in the batched FP32 form (per-lane
power-of-two exponents, FP64 endpoints and gradient accumulation).

One step = forward Gram G = k_hat(X_a, Y_b) over all 16,384 pairs x 65,536 cells, then the
adjoint: d(sum_ab W_ab G_ab)/dX and /dY for a fixed seeded upstream gradient W.
Metric: Goursat cell-updates per second of the fwd+bwd step, counting each of the Gram's
1.07e9 cells once (value = cells / step time), plus the step's milliseconds.
Timing: per-step CUDA events on the launching stream; a 256 MiB buffer is written between
steps (outside the events) so every step starts with a cold L2.

Also reported: the forward-only rate, the FP64 plain wavefront of the same Gram, the roofline of
the dominant kernel (the adjoint, FP32 ALU bound), the end-to-end rate through the public API
with host buffers, and the CPU oracle on a bounded sample.  ``--impl reference`` times the CPU
oracle alone.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

NX = NY = 128
L = 257
D = 8
DEGREE = 6
CELLS_PER_PAIR = (L - 1) * (L - 1)
CELLS = NX * NY * CELLS_PER_PAIR
PARTS = ("f32", "ckpt", "fwd", "f64", "e2e", "osc", "long", "uneven", "mmd", "acc", "cpu")
SM_COUNT = 152
FP32_LANES = 128
SM_MAX_MHZ = 2070.0


def flops_per_cell(N: int, d: int) -> int:
    """Algorithmic FLOPs of one polynomial-approximation cell update (2 per multiply-add):
    both edges' Toeplitz convolutions (N+1)(N+2), Hankel couplings 2N(N+1) and their e_n
    scalings 2(N+1), the N terms of e_m = M^m/m!, and the d-term inner product M_ij."""
    fma = (N + 1) * (N + 2) + 2 * N * (N + 1) + 2 * (N + 1) + N + d
    return 2 * fma


def adjoint_core_fma(N: int) -> int:
    """Multiply-adds of one cell's adjoint map: weights 2(N+1), Toeplitz transposes (N+1)(N+2),
    Hankel couplings 2N(N+1), and dk/dM with its recomputed Hankel sums 3N^2 + 4N."""
    return 2 * (N + 1) + (N + 1) * (N + 2) + 2 * N * (N + 1) + 3 * N * N + 4 * N


def tape_adjoint_flops_per_cell(N: int) -> int:
    """Algorithmic FLOPs of one cell of the tape adjoint kernel (2 per multiply-add): the adjoint
    map plus the N terms of e_m = M^m/m! rebuilt from the recorded M.  The forward cell is not
    recomputed and the d-term contractions run in the separate contraction kernel."""
    return 2 * (adjoint_core_fma(N) + N)


def contract_bytes_per_cell(esize: int = 4) -> int:
    """Algorithmic DRAM bytes per cell of the contraction kernel: one dk/dM element read (the
    increments it multiplies are re-read from L1/L2 and counted per pair, not per cell)."""
    return esize


def tape_steps(points: int) -> int:
    """Warp steps of one pair of `points`-point paths in the wavefront schedule (strips of 32 rows
    overlapping with period max(cols, 32))."""
    rows = cols = points - 1
    nstrips = (rows + 31) // 32
    return (nstrips - 1) * max(cols, 32) + (rows - 1 - 32 * (nstrips - 1)) + cols


def tape_adjoint_bytes(pairs: int, points: int, N: int = DEGREE) -> int:
    """Algorithmic DRAM bytes of one tape-adjoint launch: each warp step reads a 32-lane tape step
    (a, b, exponent, M padded to 16 B per lane) and writes 32 dk/dM values."""
    row = ((2 * (N + 1) + 2) * 4 + 15) // 16 * 16
    return pairs * tape_steps(points) * 32 * (row + 4)


# DRAM traffic of bwd_tape_kernel<float,6> per launch from one ncu capture on 64x64 pairs of
# 129-point paths (read 4.605319 GB + write 0.333258 GB), as a multiple of that launch's
# algorithmic bytes.  The traffic scales with the tape, so the bench launch's traffic is this ratio
# times its own algorithmic bytes.  Valid only while the kernel is unchanged since that capture.
NCU_TAPE_TRAFFIC_RATIO = (4.605319e9 + 0.333258e9) / tape_adjoint_bytes(64 * 64, 129)
HBM_GBS = 6681.2  # measured copy bandwidth of this GB300 pool


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--nx", type=int, default=NX,
                    help="paths per side (a smaller Gram of the same paths, for profiling runs)")
    ap.add_argument("--len", type=int, default=L,
                    help="points per path (shorter paths, for profiling runs that must hold only a few GB)")
    ap.add_argument("--parts", default=",".join(PARTS),
                    help="comma list: f32 (headline fwd+bwd step), ckpt (checkpointing adjoint), fwd (forward "
                         "only), f64 (FP64 forward), e2e, osc (oscillatory pairs), long (one pair of 16385-point paths), "
                         "uneven (uneven batch), mmd "
                         "(MMD^2 fwd+bwd, permutation test), acc (accuracy report: MAPE per order / refinement), cpu")
    args = ap.parse_args()
    args.parts = set(args.parts.split(","))
    if args.no_cpu_baseline:
        args.parts.discard("cpu")
    return args


def max_over_ranks(ms: float, dist, device) -> float:
    """The slowest rank's timed milliseconds (every rank gets it); `ms` itself with one rank."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(cells_per_rank: int, world: int, steps: int, total_ms: float) -> float:
    """Whole-job cell-updates/s: every rank solves its own Gram of `cells_per_rank` cells per step
    (weak scaling), and the job takes the slowest rank's time."""
    return cells_per_rank * world * steps / (total_ms / 1e3)


def workload(rank: int, n: int = NX, points: int = L):
    from paper_2502_08470_gb300 import workloads as W
    X = W.brownian(NX, points, D, seed=3 + 1000 * rank)[:n]
    Y = W.brownian(NY, points, D, seed=4 + 1000 * rank)[:n]
    return X, Y


class ClockSampler:
    """nvidia-smi clock / throttle samples taken while the timed region runs."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        # SK_CLOCKS_CSV keeps the raw samples where the caller wants them; else a temporary file,
        # removed once summarised
        self.keep = bool(os.environ.get("SK_CLOCKS_CSV"))
        self.path = os.environ.get("SK_CLOCKS_CSV") or os.path.join(tempfile.gettempdir(),
                                                                     f"sk_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self):
        lines = []
        if os.path.exists(self.path):
            with open(self.path) as f:
                lines = f.readlines()
            if not self.keep:
                os.remove(self.path)
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sms, maxs, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sms.append(float(parts[1]))
                maxs.append(float(parts[2]))
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sms) if sms else None,
                "sm_max_mhz": max(maxs) if maxs else None,
                "reasons": sorted(reasons), "samples": len(sms)}


def cpu_fwd_bwd(X, Y, points=L):
    """The FP64 oracle as it stands on one pair (prefixes of `points` points): the forward scheme
    and its complex-step gradient with respect to both paths.  Returns (cells, seconds)."""
    import oracle
    cores = os.cpu_count() or 1
    x, y = X[0][:points], Y[0][:points]
    t0 = time.perf_counter()
    oracle.kernel(x, y, "approx", DEGREE)
    oracle.grad(x, y, "approx", DEGREE, 0, threads=cores)
    return (points - 1) ** 2, time.perf_counter() - t0


def cpu_baseline(X, Y, budget_pairs=48):
    """The FP64 oracle as it stands, on bounded samples of the step: one full pair forward +
    gradient (the headline unit), and the first budget_pairs^2 pairs forward only."""
    import oracle
    cores = os.cpu_count() or 1
    cells, dt = cpu_fwd_bwd(X, Y)
    n = budget_pairs
    t0 = time.perf_counter()
    oracle.gram(list(X[:n]), list(Y[:n]), "approx", DEGREE, 0, threads=cores)
    dtf = time.perf_counter() - t0
    return {"value": cells / dt, "unit": "cell-updates/s", "cores": cores, "kind": "oracle",
            "sample": f"fwd+bwd of 1 pair (257 points, d=8, {dt:.1f} s: forward scheme + complex-step gradient "
                      f"of both paths, threads over coordinates)",
            "forward_only": {"value": n * n * CELLS_PER_PAIR / dtf, "unit": "cell-updates/s",
                             "sample": f"{n}x{n} pairs of the Gram, {dtf:.2f} s"}}


def run_reference(args, rank, world):
    import torch.distributed as dist
    if rank != 0:
        return
    X, Y = workload(0)
    cores = os.cpu_count() or 1
    for _ in range(args.warmup):
        cpu_fwd_bwd(X, Y, 65)
    cells = secs = 0.0
    for _ in range(args.steps):
        c, t = cpu_fwd_bwd(X, Y, 129)
        cells += c
        secs += t
    value = cells / secs
    ms = CELLS / value * 1e3
    sample = "per step: fwd + complex-step gradient of one pair of 129-point prefixes (128x128 cells)"
    line = {"impl": "reference",
            "metric": "Goursat cell-updates/s of the fwd+bwd Gram step (polynomial approximation N=6, 128x128 Gram)",
            "value": value, "unit": "cell-updates/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": "gram128: 128x128 Brownian paths, 257 points, d=8",
                                            "sample": sample, "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": value, "unit": "cell-updates/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "cell-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    del dist


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    import torch
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    if args.impl == "reference":
        run_reference(args, rank, world)
        if dist is not None:
            dist.barrier()
            dist.destroy_process_group()
        return

    from paper_2502_08470_gb300 import sigkernel as sk
    from paper_2502_08470_gb300 import workloads as W
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    nx = args.nx
    npts = args.len
    cells = nx * nx * (npts - 1) ** 2
    X, Y = workload(rank, nx, npts)
    Xt = torch.tensor(X, device=dev)
    Yt = torch.tensor(Y, device=dev)
    G = torch.empty(nx, nx, dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)

    Wt = torch.tensor(np.random.default_rng(11 + rank).standard_normal((nx, nx)), device=dev)
    opts = dict(scheme="approx", degree=DEGREE, sort=False)

    tape_buf = [None]

    def run(compute, steps, warmup, backward=True, tape=True):
        """Timed fwd(+bwd) steps; returns per-step ms, forward-kernel ms, adjoint-kernel ms, wall s.
        With `tape` the forward records the cell inputs and the adjoint replays them."""
        ws = sk.gram_workspace(Xt, Yt, scheme="approx", degree=DEGREE, compute=compute)

        def step(timed):
            if backward and tape:
                _, tape_buf[0] = sk.sigkernel_forward_tape(Xt, Yt, compute=compute, workspace=ws, out=G,
                                                           tape=tape_buf[0], time_kernel=timed, **opts)
            else:
                sk.sigkernel_gram(Xt, Yt, compute=compute, workspace=ws, out=G, time_kernel=timed, **opts)
            kf = sk.last_kernel_ms() if timed else None
            kb = None
            ev = None
            if backward:
                if timed:
                    ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                    ev[0].record()
                if tape:
                    sk.sigkernel_backward_tape(tape_buf[0], Wt, Xt, Yt, compute=compute, time_kernel=timed, **opts)
                else:
                    sk.sigkernel_backward(Wt, Xt, Yt, compute=compute, time_kernel=timed, **opts)
                kb = sk.last_kernel_ms() if timed else None
                if timed:
                    ev[1].record()
            return kf, kb, ev

        for _ in range(warmup):
            step(False)
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        step_ms, kf_ms, kb_ms, bc_ms = [], [], [], []
        t_wall = time.perf_counter()
        for _ in range(steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            kf, kb, ev = step(True)
            e1.record()
            e1.synchronize()
            step_ms.append(e0.elapsed_time(e1))
            if ev is not None:
                bc_ms.append(ev[0].elapsed_time(ev[1]))
            kf_ms.append(kf)
            if kb is not None:
                kb_ms.append(kb)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t_wall
        if dist is not None:
            dist.barrier()
        run.backward_call_ms = bc_ms
        return step_ms, kf_ms, kb_ms, wall

    line = {}
    fpc = flops_per_cell(DEGREE, D)
    bpc = tape_adjoint_flops_per_cell(DEGREE)
    peak = SM_COUNT * FP32_LANES * 2 * SM_MAX_MHZ * 1e6 / 1e12
    import oracle
    rng = np.random.default_rng(0)
    pa = rng.integers(0, nx, 16)
    pb = rng.integers(0, nx, 16)

    # headline: fwd + bwd step, batched FP32 form
    with ClockSampler(local) as clk:
        step_ms, kf_ms, kb_ms, wall = run("f32", args.steps, max(args.warmup, 3))
    clocks = clk.summary()
    total_ms = max_over_ranks(float(sum(step_ms)), dist, dev)
    ms_per_step = total_ms / args.steps
    value = job_throughput(cells, world, args.steps, total_ms)
    g32 = G.cpu().numpy()[pa, pb]
    status = sk.device_status()
    kf = statistics.mean(kf_ms)
    kb = statistics.mean(kb_ms)
    bcall = statistics.mean(run.backward_call_ms) if run.backward_call_ms else None
    ach_b = bpc * cells / (kb / 1e3) / 1e12
    ach_f = fpc * cells / (kf / 1e3) / 1e12
    ref = oracle.pairs(list(X), list(Y), pa, pb, "approx", DEGREE)
    mape = {"f32": float(np.mean(np.abs(g32 - ref) / np.abs(ref))), "sample": "16 sampled Gram entries"}
    line.update({
        "metric": "Goursat cell-updates/s of the fwd+bwd Gram step (polynomial approximation N=6, 128x128 Gram, "
                  "batched FP32, forward tape)",
        "value": value, "unit": "cell-updates/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"gram{nx}: X, Y = {nx} Brownian paths each, {npts} points, d=8, N(0,1/{npts - 1}) "
                               "increments; "
                               "step = forward Gram + adjoint for a seeded upstream gradient",
                   "scheme": "polynomial approximation", "degree": DEGREE, "dyadic": 0,
                   "cells_per_step": cells, "pairs_per_step": nx * nx,
                   "l2": "256 MiB buffer written between timed steps (outside the events)",
                   "tape_gb": round(tape_buf[0].numel() / 1e9, 2),
                   "parallelism": f"weak scaling, one independent {nx}x{nx} Gram per GPU ({world} GPUs)"},
        "roofline": {"bound": "alu", "achieved": ach_b, "peak": peak, "unit": "TFLOP/s", "frac": ach_b / peak,
                     "traffic": NCU_TAPE_TRAFFIC_RATIO * tape_adjoint_bytes(nx * nx, npts),
                     "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of one 64x64x129-point "
                                       "launch, scaled by algorithmic tape bytes to this launch",
                     "algorithmic_bytes": tape_adjoint_bytes(nx * nx, npts),
                     "hbm_gbs": tape_adjoint_bytes(nx * nx, npts) / (kb / 1e3) / 1e9,
                     "hbm_frac_of_measured": tape_adjoint_bytes(nx * nx, npts) / (kb / 1e3) / 1e9 / HBM_GBS,
                     "kernel": "bwd_tape_kernel<float,6> (adjoint wavefront from the tape)",
                     "kernel_ms": kb,
                     "flops_per_cell": bpc,
                     "peak_source": "152 SMs x 128 FP32 lanes x 2 FLOP x 2070 MHz (derived, nominal clocks)"},
        "forward_kernel": {"kernel": "fwd_poly_kernel<float,6,6,false> (recording the tape)", "kernel_ms": kf,
                           "achieved_tflops": ach_f,
                           "frac": ach_f / peak, "flops_per_cell": fpc,
                           "cell_updates_per_s": cells / (kf / 1e3)},
        "backward_call": {"ms": bcall, "adjoint_kernel_ms": kb,
                          "rest_ms": (bcall - kb) if bcall is not None else None,
                          "rest": "increments, dk/dM contraction kernel, gradient conversions"},
        # forward: 2 increments + wavefront; adjoint: 2 increments + adjoint + contraction + 2 gradient conversions
        "gpu_launches": 9 * args.steps,
        "clocks": clocks, "device_status": status, "wall_s_timed_region": wall,
    })

    if "ckpt" in args.parts:  # the same step with the checkpointing adjoint (no tape)
        sc, kfc, kbc, _ = run("f32", max(2, min(3, args.steps)), 1, tape=False)
        line["checkpoint_adjoint"] = {"value": cells / (statistics.mean(sc) / 1e3), "unit": "cell-updates/s",
                                      "ms_per_step": statistics.mean(sc), "forward_kernel_ms": statistics.mean(kfc),
                                      "adjoint_kernel_ms": statistics.mean(kbc)}
    tape_buf[0] = None
    torch.cuda.empty_cache()

    if "fwd" in args.parts:  # forward only (the Gram alone)
        sf, kff, _, _ = run("f32", args.steps, 2, backward=False)
        line["forward_only"] = {"value": cells / (statistics.mean(sf) / 1e3), "unit": "cell-updates/s",
                                "ms_per_step": statistics.mean(sf), "kernel_ms": statistics.mean(kff)}

    if "f64" in args.parts:  # FP64 plain wavefront of the same Gram (a few steps)
        s64, k64, _, _ = run("f64", max(2, min(3, args.steps)), 1, backward=False)
        g64 = G.cpu().numpy()[pa, pb]
        k64avg = statistics.mean(k64)
        mape["f64"] = float(np.mean(np.abs(g64 - ref) / np.abs(ref)))
        line["fp64_plain_wavefront"] = {"value": cells / (statistics.mean(s64) / 1e3), "unit": "cell-updates/s",
                                        "kernel_ms": k64avg, "achieved_tflops": fpc * cells / (k64avg / 1e3) / 1e12,
                                        "peak_tflops_nominal": 1.25}
    line["mape_vs_fp64_oracle"] = mape

    if "e2e" in args.parts:  # end to end through the public API with pinned host buffers
        Xh = torch.tensor(X).pin_memory()
        Yh = torch.tensor(Y).pin_memory()
        Wh = Wt.cpu().pin_memory()
        Gh = torch.empty(nx, nx, dtype=torch.float64).pin_memory()
        gXh = torch.empty(nx * npts, D, dtype=torch.float64).pin_memory()
        gYh = torch.empty(nx * npts, D, dtype=torch.float64).pin_memory()
        ws = sk.gram_workspace(Xt, Yt, scheme="approx", degree=DEGREE, compute="f32")
        Wd = torch.empty_like(Wt)
        e2e_ms = []
        for it in range(args.warmup + args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            Xt.copy_(Xh, non_blocking=True)
            Yt.copy_(Yh, non_blocking=True)
            Wd.copy_(Wh, non_blocking=True)
            _, tape_buf[0] = sk.sigkernel_forward_tape(Xt, Yt, compute="f32", workspace=ws, out=G, tape=tape_buf[0],
                                                       **opts)
            gX, gY = sk.sigkernel_backward_tape(tape_buf[0], Wd, Xt, Yt, compute="f32", **opts)
            Gh.copy_(G, non_blocking=True)
            gXh.copy_(gX, non_blocking=True)
            gYh.copy_(gY, non_blocking=True)
            e1.record()
            e1.synchronize()
            if it >= args.warmup:
                e2e_ms.append(e0.elapsed_time(e1))
        line["e2e"] = {"value": cells * world / (statistics.mean(e2e_ms) / 1e3), "unit": "cell-updates/s",
                       "h2d_bytes_per_step": int((Xh.numel() + Yh.numel() + Wh.numel()) * 8),
                       "d2h_bytes_per_step": int((Gh.numel() + gXh.numel() + gYh.numel()) * 8),
                       "ms_per_step": statistics.mean(e2e_ms)}
        tape_buf[0] = None

    tape_buf[0] = None
    torch.cuda.empty_cache()

    def timed_steps(fn, steps, warmup):
        """Per-call milliseconds (CUDA events on the current stream, L2 flushed before each call)."""
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        ms = []
        for _ in range(steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        return statistics.mean(ms)

    if "osc" in args.parts:  # 64 pairs of 1025-point oscillatory paths, d=4 (few long pairs: strip pipeline)
        Xo = torch.tensor(W.oscillatory(64, 1025, 4, seed=5 + 1000 * rank), device=dev)
        Yo = torch.tensor(W.oscillatory(64, 1025, 4, seed=6 + 1000 * rank), device=dev)
        io = torch.arange(64, dtype=torch.int64, device=dev)
        cells_o = 64 * 1024 * 1024
        osc = {"workload": "64 pairs, 1025 points on [0,1], d=4, sin(w t + phi) + N(0,1e-3), w ~ U(10,200)"}
        for scheme, N, lam, comp in (("interp", 8, 0, "f32"), ("interp", 8, 0, "f64"), ("fd1", 2, 0, "f32"),
                                     ("fd1", 2, 2, "f32"), ("fd1", 2, 4, "f32"), ("fd1", 2, 6, "f32"),
                                     ("fd2", 2, 4, "f32"), ("fd_implicit", 2, 4, "f32")):
            o = torch.empty(64, dtype=torch.float64, device=dev)
            f = lambda: sk.sigkernel_pairs(Xo, Yo, io, io, scheme=scheme, degree=N, dyadic=lam, compute=comp, out=o)
            t = timed_steps(f, 1 if lam == 6 else 3, 1)
            key = f"{scheme}{N if scheme == 'interp' else ''}_lam{lam}_{comp}"
            osc[key] = {"ms": t, "cell_updates_per_s": cells_o / (t / 1e3),
                        "sub_cell_updates_per_s": cells_o * 4 ** lam / (t / 1e3)}
            if key == "interp8_lam0_f32":
                o32 = o.clone()
            if key == "interp8_lam0_f64":
                osc["interp8_f32_mape_vs_fp64_gpu"] = float(((o32 - o).abs() / o.abs()).mean())
        line["oscillatory"] = osc
        del Xo, Yo

    if "long" in args.parts:  # one pair of 16385-point paths, d=4: parallelism inside a single pair
        Xl = torch.tensor(W.brownian(1, 16385, 4, seed=11 + 1000 * rank), device=dev)
        Yl = torch.tensor(W.brownian(1, 16385, 4, seed=12 + 1000 * rank), device=dev)
        il = torch.zeros(1, dtype=torch.int64, device=dev)
        ol = torch.empty(1, dtype=torch.float64, device=dev)
        cells_l = 16384 * 16384
        t_grid = timed_steps(lambda: sk.sigkernel_pairs(Xl, Yl, il, il, compute="f32", out=ol), 2, 1)
        line["long_pair"] = {"workload": "1 pair of 16385-point Brownian paths, d=4, approx N=6, FP32: the pair's "
                                         "512 strips swept by a ring of 32 co-resident 16-warp blocks",
                             "cells": cells_l, "ms": t_grid, "cell_updates_per_s": cells_l / (t_grid / 1e3)}
        del Xl, Yl

    if "uneven" in args.parts:  # 4096 pairs, lengths log-uniform in [64, 4096], d=16, BF16: autotuned + graph
        Xs = W.uneven(4096, 64, 4096, 16, seed=6 + 1000 * rank)
        Ys = W.uneven(4096, 64, 4096, 16, seed=7 + 1000 * rank)
        PX = sk.Paths.from_list(Xs, dtype=torch.bfloat16)
        PY = sk.Paths.from_list(Ys, dtype=torch.bfloat16)
        cells_u = float(sum((len(x) - 1) * (len(y) - 1) for x, y in zip(Xs, Ys)))
        iu = torch.arange(4096, dtype=torch.int64, device=dev)
        ou = torch.empty(4096, dtype=torch.float64, device=dev)
        sk.autotune_clear()
        shape, tuned_ms = sk.autotune(PX, PY, iu, iu, compute="f32", trials=1)
        t_tuned = timed_steps(lambda: sk.sigkernel_pairs(PX, PY, iu, iu, compute="f32", out=ou), 3, 1)
        t_one = timed_steps(lambda: sk.sigkernel_pairs(PX, PY, iu, iu, compute="f32", out=ou,
                                                       strip_pipeline=False), 2, 1)
        graph = torch.cuda.CUDAGraph()
        gs = torch.cuda.Stream()
        with torch.cuda.stream(gs):
            with torch.cuda.graph(graph, stream=gs):
                sk.sigkernel_pairs(PX, PY, iu, iu, compute="f32", out=ou)
        t_graph = timed_steps(graph.replay, 3, 1)
        line["uneven_batch"] = {
            "workload": "4096 pairs, lengths log-uniform in [64,4096], d=16, BF16 points, approx N=6, FP32 cells",
            "cells": cells_u, "autotuned_shape": shape, "ms": t_tuned,
            "cell_updates_per_s": cells_u / (t_tuned / 1e3), "graph_replay_ms": t_graph,
            "graph_cell_updates_per_s": cells_u / (t_graph / 1e3), "one_warp_per_pair_ms": t_one}
        sk.autotune_clear()
        del PX, PY, graph

    if "mmd" in args.parts:  # MMD^2 fwd+bwd: 256 + 256 paths, 513 points, d=32, FP32, checkpointing adjoint
        Am = torch.tensor(W.brownian(256, 513, 32, seed=7 + 1000 * rank), device=dev)
        Bm = torch.tensor(W.brownian(256, 513, 32, seed=8 + 1000 * rank, drift=0.5, vol=1.2), device=dev)
        cells_m = (256 * 257 // 2 * 2 + 256 * 256) * 512 * 512
        t_f = timed_steps(lambda: sk.sigkernel_mmd2(Am, Bm, degree=6, compute="f32"), 2, 1)
        t_fb = timed_steps(lambda: sk.sigkernel_mmd2(Am, Bm, degree=6, compute="f32", grads=True), 2, 1)
        labels = sk.split_labels(1000, 256, 256, seed=9 + rank)
        ws_t = sk.mmd2_test_workspace(Am, Bm, 1000, compute="f32")
        out_t = torch.empty(1002, dtype=torch.float64, device=dev)
        t_test = timed_steps(lambda: sk.sigkernel_mmd2_test(Am, Bm, labels=labels, compute="f32", workspace=ws_t,
                                                            out=out_t), 2, 1)
        line["mmd2"] = {"workload": "256 + 256 paths, 513 points, d=32 (Brownian vs drift 0.5, vol 1.2), approx N=6, "
                                    "FP32, symmetric K_AA/K_BB + K_AB, tiled M; gradients from forward tapes in "
                                    "chunks of pairs (tape <= 48 GiB per chunk)",
                        "cells": cells_m, "forward_ms": t_f, "fwd_bwd_ms": t_fb,
                        "forward_cell_updates_per_s": cells_m / (t_f / 1e3),
                        "fwd_bwd_cell_updates_per_s": cells_m / (t_fb / 1e3),
                        "permutation_test_1000_ms": t_test,
                        "permutation_test_p_value": out_t[1].item()}
        del Am, Bm, ws_t

    if "acc" in args.parts and rank == 0:  # MAPE per order / refinement against a converged FP64 solution
        from paper_2502_08470_gb300 import accuracy

        def sig3(rep):
            return {L: {k: (round(v, 12) if k == "truth_check" else {o: float(f"{e:.3g}") for o, e in v.items()})
                        for k, v in row.items()} for L, row in rep["lengths"].items()}
        line["accuracy"] = {"truth": "interpolation N=12, lambda=3, FP64 (checked against approximation N=16)",
                            "unit": "MAPE in percent; keys: order N (approx, interp) or dyadic lambda (fd*)"}
        for kind, lengths in (("sin", (10, 50, 100, 200)), ("brownian", (10, 50, 200))):
            line["accuracy"][kind] = {c: sig3(accuracy.report(kind, lengths=lengths, compute=c))
                                      for c in ("f64", "f32")}

    if rank == 0:
        if "cpu" in args.parts:
            line["cpu_baseline"] = cpu_baseline(X, Y)
        print(json.dumps(line))
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
