#!/usr/bin/env python3
"""Throughput benchmark of the signature-kernel Gram path on GB300.

Workload ("gram128"): X and Y are 128 Brownian paths each on [0, 1], 257 points, d = 8,
increments N(0, 1/256) per coordinate (seeds 3 and 4; other ranks use their own seeds), solved
with the polynomial approximation scheme of order 6 in the batched FP32 form (per-lane
power-of-two exponents, FP64 endpoints and gradient accumulation).

One step = forward Gram G = k_hat(X_a, Y_b) over all 16,384 pairs x 65,536 cells, recording the
tape the adjoint reads, then the adjoint: d(sum_ab W_ab G_ab)/dX and /dY for a fixed seeded
upstream gradient W.
Metric: Goursat cell-updates per second of the fwd+bwd step, counting each of the Gram's
1.07e9 cells once (value = cells / step time), plus the step's milliseconds.
Timing: per-step CUDA events on the launching stream; a 256 MiB buffer is written between
steps (outside the events) so every step starts with a cold L2.

Also reported (parts, --parts): the public sigkernel_backward and autograd paths, the forward
alone, the FP64 plain wavefront forward and fwd+bwd, the end-to-end rate through the public API
with host buffers, the single-pair latency of the plain method, the FD schemes on the same Gram,
the oscillatory, long-pair, uneven-batch and MMD workloads, the accuracy study, and the CPU
oracle.  Roofline fractions divide by peaks measured in the same run: the FP32 / FP64 FMA rate
(sigkernel_fma_peak) and the HBM copy bandwidth of MEASURED_PEAKS.json.

The FP64 oracle runs only in the CPU-baseline leg (`cpu` part), on rank 0: it computes the
sampled outputs that every GPU part kept, which gives each part's MAPE against the oracle, and
its own timing is the CPU baseline.  ``--impl reference`` times the CPU oracle alone.
"""
from __future__ import annotations

import argparse
import json
import os
import socket
import statistics
import subprocess
import sys
import tempfile
import time
from math import factorial

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

NX = NY = 128
L = 257
D = 8
DEGREE = 6
CELLS_PER_PAIR = (L - 1) * (L - 1)
CELLS = NX * NY * CELLS_PER_PAIR
PARTS = ("f32", "api", "fwd", "f64", "e2e", "single", "gram_fd", "osc", "long", "uneven", "mmd", "acc", "cpu")
METRIC = ("Goursat cell-updates/s of the fwd+bwd Gram step (polynomial approximation N=6, 128x128 Gram of "
          "257-point paths, d=8)")
FALLBACK_HBM_GBS = 6800.0  # the profiling recipe's fallback when MEASURED_PEAKS.json is absent
SM_COUNT, FP32_LANES, SM_MAX_MHZ = 152, 128, 2070.0  # nominal, for context only


def flops_per_cell(N: int, d: int) -> int:
    """Algorithmic FLOPs of one polynomial-approximation cell update (2 per multiply-add), as the
    kernels compute it: with e_0 = 1 every output c_n = e_n (c_0 + H_n) + sum_{1<=k<n} c_k e_{n-k}
    + c_n costs N multiply-adds for the corner term plus Hankel coupling (n = 0..N), n - 1 for the
    rest of the Toeplitz convolution and one for the scaling (n >= 1), on both edges; then the N
    terms of e_m = M^m/m! and the d-term inner product M_ij.  (Counting the products with e_0 and
    each sum's first product, as a literal reading of the update does, gives 336 instead of 280
    at N = 6, d = 8.)"""
    fma = 2 * N * (N + 1) + N * (N - 1) + 2 * N + N + d
    return 2 * fma


def tape_forward_flops_per_cell(N: int, d: int) -> int:
    """The forward cell plus the 2N derivatives d a'_n/dM, d b'_n/dM it records on the tape (one
    multiply-add each but the first of each edge, which is the n = 1 coupling sum itself)."""
    return flops_per_cell(N, d) + 2 * 2 * (N - 1)


def adjoint_edge_fma(N: int) -> int:
    """Multiply-adds of one cell's edge adjoints: Hankel weights g_n e_n (n >= 1) on both edges 2N,
    Toeplitz transposes N(N+1) (each sum starts from its e_0 term), Hankel couplings 2N(N+1)."""
    return 2 * N + N * (N + 1) + 2 * N * (N + 1)


def tape_adjoint_flops_per_cell(N: int) -> int:
    """Algorithmic FLOPs of one cell of the tape adjoint kernel (2 per multiply-add): the edge
    adjoints, dk/dM from the 2N recorded derivatives, and the N terms of e_m = M^m/m! rebuilt from
    the recorded M.  The d-term contractions run in the separate contraction kernel."""
    return 2 * (adjoint_edge_fma(N) + 2 * N + N)


def tape_row_bytes(N: int, esize: int = 4) -> int:
    """One lane's tape row of the approximation scheme: 2N derivatives, the exponent and M."""
    return (2 * N + 2) * esize


def tape_steps(points: int) -> int:
    """Warp steps of one pair of `points`-point paths in the wavefront schedule (strips of 32 rows
    overlapping with period max(cols, 32))."""
    rows = cols = points - 1
    nstrips = (rows + 31) // 32
    return (nstrips - 1) * max(cols, 32) + (rows - 1 - 32 * (nstrips - 1)) + cols


def tape_forward_bytes(pairs: int, points: int, N: int = DEGREE, esize: int = 4) -> int:
    """Algorithmic DRAM bytes the tape forward writes: one row per lane per warp step."""
    return pairs * tape_steps(points) * 32 * tape_row_bytes(N, esize)


def tape_adjoint_bytes(pairs: int, points: int, N: int = DEGREE, esize: int = 4) -> int:
    """Algorithmic DRAM bytes of one tape-adjoint launch: each warp step reads a 32-lane tape step
    and writes 32 dk/dM values."""
    return pairs * tape_steps(points) * 32 * (tape_row_bytes(N, esize) + esize)


def load_hbm_peak():
    """(GB/s, source): the measured copy bandwidth of MEASURED_PEAKS.json, else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            v = float(json.load(f)["hbm_gbs"])
        return v, "measured (MEASURED_PEAKS.json copy bandwidth)"
    except (OSError, ValueError, KeyError, TypeError):
        return FALLBACK_HBM_GBS, "fallback (profiling recipe, MEASURED_PEAKS.json absent)"


# DRAM traffic (ncu dram__bytes_read.sum + dram__bytes_write.sum) of one launch, as a multiple of
# that launch's algorithmic bytes, from captures of the current kernels on 48 x 48 pairs of
# 129-point paths (profiles/*_gram48x129.md): both kernels' traffic is per warp step, so it
# scales with the steps of the bench's Gram.  None when no capture of the current kernel exists.
NCU_TRAFFIC_RATIO = {"bwd_tape_kernel<float,6,false>": (2.270 + 0.185) / 2.402,
                     "fwd_poly_kernel<float,6,6,false,1,false,true,true>": (2.207 + 0.161) / 2.242}


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
    ap.add_argument("--mmd-n", type=int, default=256,
                    help="paths per sample of the mmd part (fewer, for profiling runs that must hold only a few GB)")
    ap.add_argument("--mmd-forward-only", action="store_true",
                    help="mmd part: the forward alone (profiling runs that must not hold a gradient tape)")
    ap.add_argument("--parts", default=",".join(PARTS),
                    help="comma list: f32 (headline fwd+bwd step), api (sigkernel_backward, autograd, checkpointing "
                         "adjoint), fwd (forward only), f64 (FP64 forward and fwd+bwd), e2e, single (one pair of "
                         "33-point paths), gram_fd (FD schemes on the Gram), osc (oscillatory pairs), long (one pair "
                         "of 16385-point paths), uneven (uneven batch), mmd (MMD^2 fwd+bwd, permutation test), acc "
                         "(accuracy report), cpu (the oracle: CPU baseline and every part's MAPE)")
    args = ap.parse_args()
    args.parts = set(args.parts.split(","))
    if args.no_cpu_baseline:
        args.parts.discard("cpu")
    return args


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def ensure_world(args) -> None:
    """--gpus N without a launcher: start N ranks with torch.distributed.run on this node (and
    exit with their status).  Under a launcher, WORLD_SIZE must equal N."""
    world = os.environ.get("WORLD_SIZE")
    if world is None and args.gpus > 1:
        cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={args.gpus}",
               "--master-addr=127.0.0.1", f"--master-port={_free_port()}", os.path.abspath(__file__)] + sys.argv[1:]
        sys.exit(subprocess.call(cmd))
    if world is not None and int(world) != args.gpus:
        sys.exit(f"bench.py: --gpus {args.gpus} but WORLD_SIZE={world}")


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
        self.f = None
        self.error = None
        # SK_CLOCKS_CSV keeps the raw samples where the caller wants them; else a temporary file,
        # removed once summarised
        self.keep = bool(os.environ.get("SK_CLOCKS_CSV"))
        self.path = os.environ.get("SK_CLOCKS_CSV") or os.path.join(tempfile.gettempdir(),
                                                                     f"sk_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            parent = os.path.dirname(self.path)
            if parent:
                os.makedirs(parent, exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError as e:
            self.error = f"{type(e).__name__}: {e}"
            self.proc = None
            if self.f is not None:
                self.f.close()
                self.f = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.f is not None:
            self.f.close()
            self.f = None

    def summary(self):
        lines = []
        if os.path.exists(self.path):
            with open(self.path) as f:
                lines = f.readlines()
            if not self.keep:
                os.remove(self.path)
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [f"no samples: {self.error or 'nvidia-smi'}"]}
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


# ---------------------------------------------------------------------------------------------
# The CPU oracle (only here and in the reference arm).
# ---------------------------------------------------------------------------------------------
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


def oracle_samples(samples):
    """Runs the oracle on every part's sampled pairs.  `samples` maps a part's name to a dict with
    the paths xs, ys (lists of float64 arrays: the exact numbers the GPU saw), the pairs pa, pb,
    the scheme, N, lambda and the GPU values `gpu` (one per pair, or a dict of several columns);
    returns ({name: MAPE dict}, oracle seconds, oracle cells)."""
    import oracle
    cores = os.cpu_count() or 1
    out, secs, cells = {}, 0.0, 0.0
    for name, s in samples.items():
        t0 = time.perf_counter()
        ref = oracle.pairs(s["xs"], s["ys"], s["pa"], s["pb"], s["scheme"], s["N"], s["lam"], threads=cores)
        secs += time.perf_counter() - t0
        cells += float(sum((len(s["xs"][a]) - 1) * (len(s["ys"][b]) - 1) for a, b in zip(s["pa"], s["pb"])))
        gpu = s["gpu"] if isinstance(s["gpu"], dict) else {"value": s["gpu"]}
        keep = np.abs(ref) >= 1e-3  # relative error is not defined near a zero of the kernel
        m = {}
        for col, g in gpu.items():
            rel = np.abs(np.asarray(g, dtype=np.float64) - ref)[keep] / np.abs(ref[keep])
            m[col] = {"mape": float(rel.mean()) if rel.size else None,
                      "max_rel": float(rel.max()) if rel.size else None}
        m["pairs"] = int(len(ref))
        if not keep.all():
            m["excluded_near_zero"] = int((~keep).sum())
        m["scheme"] = f"{s['scheme']} N={s['N']} lambda={s['lam']}"
        out[name] = m
    return out, secs, cells


def cpu_baseline(X, Y, samples):
    """The FP64 oracle as it stands, timed on the host cores: fwd+bwd of one full pair (the
    headline unit: forward scheme and complex-step gradient), and the forward rate over every
    part's sampled pairs, which also gives each part's MAPE against the oracle."""
    cores = os.cpu_count() or 1
    cells, dt = cpu_fwd_bwd(X, Y)
    mape, secs, fcells = oracle_samples(samples)
    return {"value": cells / dt, "unit": "cell-updates/s", "cores": cores, "kind": "oracle",
            "sample": f"fwd+bwd of 1 pair (257 points, d=8, {dt:.1f} s: forward scheme + complex-step gradient "
                      f"of both paths, threads over coordinates)",
            "forward_only": {"value": fcells / secs if secs > 0 else None, "unit": "cell-updates/s",
                             "sample": f"the sampled pairs of every part ({fcells:.3g} cells, {secs:.1f} s, threads "
                                       f"over pairs)"}}, mape


def run_reference(args, rank, world):
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
    sample = ("each step: fwd + complex-step gradient of one pair of 129-point prefixes of the workload's first pair "
              "(16,384 cells), threads over coordinates")
    line = {"impl": "reference", "metric": METRIC,
            "value": value, "unit": "cell-updates/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": secs / args.steps * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": "gram128: X, Y = 128 Brownian paths each, 257 points, d=8, N(0,1/256) increments",
                       "sample": sample, "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": value, "unit": "cell-updates/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "cell-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ---------------------------------------------------------------------------------------------
# The GPU arm.
# ---------------------------------------------------------------------------------------------
def main():
    args = parse()
    ensure_world(args)
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
    rng = np.random.default_rng(0)
    samples = {}  # part -> sampled pairs and GPU values, for the oracle leg

    def sample_gram(name, Gm, n=64, scheme="approx", N=DEGREE, lam=0, Xs=X, Ys=Y, extra=None):
        pa = rng.integers(0, Gm.shape[0], n)
        pb = rng.integers(0, Gm.shape[1], n)
        g = Gm.cpu().numpy()[pa, pb]
        gpu = {"value": g}
        if extra:
            gpu.update({k: v.cpu().numpy()[pa, pb] for k, v in extra.items()})
        samples[name] = dict(xs=list(Xs), ys=list(Ys), pa=pa, pb=pb, scheme=scheme, N=N, lam=lam, gpu=gpu)

    # measured peaks: FP32 / FP64 FMA rates (this run, with their clocks) and the HBM copy bandwidth
    with ClockSampler(local) as pclk:
        p32 = max(sk.fma_peak("f32", packed=False), sk.fma_peak("f32", packed=True))
        p64 = sk.fma_peak("f64")
    hbm_peak, hbm_src = load_hbm_peak()
    peaks = {"fp32_tflops": p32, "fp64_tflops": p64, "hbm_gbs": hbm_peak, "hbm_source": hbm_src,
             "fma_source": "sigkernel_fma_peak: independent FMA chains (FP32 scalar and two-wide, the faster), 4 x 384 "
                           "threads per SM, fastest of 5 launches, CUDA events",
             "fma_clocks": pclk.summary(),
             "fp32_nominal_tflops": SM_COUNT * FP32_LANES * 2 * SM_MAX_MHZ * 1e6 / 1e12}

    tape_buf = [None]

    def run(compute, steps, warmup, backward=True, tape=True, Xa=Xt, Ya=Yt, Wa=Wt, out=G):
        """Timed fwd(+bwd) steps; returns per-step ms, forward-kernel ms, adjoint-kernel ms, wall s.
        With `tape` the forward records the tape and the adjoint replays it; without it the backward
        is the public sigkernel_backward."""
        ws = sk.gram_workspace(Xa, Ya, scheme="approx", degree=DEGREE, compute=compute)

        def step(timed):
            if backward and tape:
                _, tape_buf[0] = sk.sigkernel_forward_tape(Xa, Ya, compute=compute, workspace=ws, out=out,
                                                           tape=tape_buf[0], time_kernel=timed, **opts)
            else:
                sk.sigkernel_gram(Xa, Ya, compute=compute, workspace=ws, out=out, time_kernel=timed, **opts)
            kf = sk.last_kernel_ms() if timed else None
            kb = None
            ev = None
            if backward:
                if timed:
                    ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                    ev[0].record()
                if tape:
                    sk.sigkernel_backward_tape(tape_buf[0], Wa, Xa, Ya, compute=compute, time_kernel=timed, **opts)
                    kb = sk.last_kernel_ms() if timed else None
                else:
                    sk.sigkernel_backward(Wa, Xa, Ya, compute=compute, **opts)
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

    def kernel_roofline(name, ms, flops, bytes_, peak_tflops, ratio_key=None):
        """ALU and HBM fractions of one kernel launch; `bound` is the larger of the two."""
        alu = flops / (ms / 1e3) / 1e12
        hbm = bytes_ / (ms / 1e3) / 1e9
        fa, fh = alu / peak_tflops, hbm / hbm_peak
        ratio = NCU_TRAFFIC_RATIO.get(ratio_key) if ratio_key else None
        r = {"kernel": name, "kernel_ms": ms, "alu_tflops": alu, "alu_frac": fa, "hbm_gbs": hbm, "hbm_frac": fh,
             "algorithmic_bytes": bytes_, "algorithmic_flops": flops,
             "traffic": ratio * bytes_ if ratio is not None else None}
        if fh > fa:
            r.update({"bound": "hbm", "achieved": hbm, "peak": hbm_peak, "unit": "GB/s", "frac": fh})
        else:
            r.update({"bound": "alu", "achieved": alu, "peak": peak_tflops, "unit": "TFLOP/s", "frac": fa})
        return r

    line = {}
    # headline: fwd + bwd step, batched FP32 form, forward tape
    with ClockSampler(local) as clk:
        step_ms, kf_ms, kb_ms, wall = run("f32", args.steps, max(args.warmup, 3))
    clocks = clk.summary()
    total_ms = max_over_ranks(float(sum(step_ms)), dist, dev)
    ms_per_step = total_ms / args.steps
    value = job_throughput(cells, world, args.steps, total_ms)
    sample_gram("f32", G)
    status = sk.device_status()
    kf = statistics.mean(kf_ms)
    kb = statistics.mean(kb_ms)
    bcall = statistics.mean(run.backward_call_ms) if run.backward_call_ms else None
    tape_gb = tape_buf[0].numel() / 1e9
    fwd_rl = kernel_roofline("m_tc_kernel<16> + fwd_poly_kernel<float,6,6,false,1,false,true,true> (forward "
                             "recording the tape, M from the tensor cores; algorithmic bytes: the tape)", kf,
                             tape_forward_flops_per_cell(DEGREE, D) * cells, tape_forward_bytes(nx * nx, npts), p32,
                             "fwd_poly_kernel<float,6,6,false,1,false,true,true>")
    bwd_rl = kernel_roofline("bwd_tape_kernel<float,6,false> (adjoint wavefront from the tape)", kb,
                             tape_adjoint_flops_per_cell(DEGREE) * cells, tape_adjoint_bytes(nx * nx, npts), p32,
                             "bwd_tape_kernel<float,6,false>")
    dominant = bwd_rl if kb >= kf else fwd_rl
    roofline = {k: dominant[k] for k in ("bound", "achieved", "peak", "unit", "frac", "traffic")}
    roofline.update({"kernel": dominant["kernel"], "kernel_ms": dominant["kernel_ms"],
                     "peak_source": "measured in this run: " + ("sigkernel_fma_peak FP32" if dominant["unit"] == "TFLOP/s"
                                                                else hbm_src),
                     "alu_frac": dominant["alu_frac"], "hbm_frac": dominant["hbm_frac"],
                     "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch on 48 x 48 "
                                       "pairs of 129-point paths, as a multiple of its algorithmic bytes, times this "
                                       "launch's algorithmic bytes" if
                     dominant["traffic"] is not None else "no ncu capture of the current kernel"})
    line.update({
        "metric": METRIC,
        "value": value, "unit": "cell-updates/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"gram{nx}: X, Y = {nx} Brownian paths each, {npts} points, d=8, N(0,1/{npts - 1}) "
                               "increments; step = forward Gram recording the tape + adjoint for a seeded upstream "
                               "gradient",
                   "scheme": "polynomial approximation", "degree": DEGREE, "dyadic": 0,
                   "cells_per_step": cells, "pairs_per_step": nx * nx,
                   "l2": "256 MiB buffer written between timed steps (outside the events)",
                   "tape_gb": round(tape_gb, 2),
                   "parallelism": f"weak scaling, one independent {nx}x{nx} Gram per GPU ({world} GPUs)"},
        "roofline": roofline,
        "kernels": {"forward_tape": fwd_rl, "adjoint": bwd_rl,
                    "backward_call": {"ms": bcall, "adjoint_kernel_ms": kb,
                                      "rest_ms": (bcall - kb) if bcall is not None else None,
                                      "rest": "increments, dk/dM contraction kernel, gradient conversions"}},
        "peaks": peaks,
        # forward: 2 increments + 2 BF16 operand splits + tensor-core M + wavefront; adjoint: 2
        # increments + adjoint + contraction + 2 gradient conversions (the ncu launch list of the
        # same command, profiles/launches_gram128.md, counts the same 12 per step)
        "gpu_launches": 12 * args.steps,
        "clocks": clocks, "device_status": status, "wall_s_timed_region": wall,
        "device": {"gpu": torch.cuda.get_device_name(local), "host_cores": os.cpu_count() or 1},
    })
    tape_buf[0] = None
    torch.cuda.empty_cache()

    if "api" in args.parts:
        # the public sigkernel_backward (chunked tapes: re-runs the forward) after a plain forward,
        # the autograd wrapper, and the checkpointing adjoint
        sa, _, _, _ = run("f32", max(2, min(3, args.steps)), 1, tape=False)
        api = {"sigkernel_backward": {"step_ms": statistics.mean(sa),
                                      "backward_call_ms": statistics.mean(run.backward_call_ms),
                                      "cell_updates_per_s": cells / (statistics.mean(sa) / 1e3),
                                      "what": "forward Gram, then sigkernel_backward (forward tapes in chunks of "
                                              "<= 64 GiB and the tape adjoint after each)"}}
        kern = sk.SigKernel("approx", DEGREE, 0, "f32")
        Xg = Xt.clone().requires_grad_(True)
        Yg = Yt.clone().requires_grad_(True)

        def ag_step():
            Gg = kern.gram(Xg, Yg)
            (Gg * Wt).sum().backward()
        ms = []
        for it in range(3 + 2):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            ag_step()
            e1.record()
            e1.synchronize()
            if it >= 2:
                ms.append(e0.elapsed_time(e1))
            Xg.grad = Yg.grad = None
        api["autograd"] = {"step_ms": statistics.mean(ms), "cell_updates_per_s": cells / (statistics.mean(ms) / 1e3),
                           "what": "SigKernel(approx, 6, f32).gram(X, Y), (G * W).sum().backward(): the forward "
                                   "keeps its tape (tape=None chooses it when it fits)"}
        del Xg, Yg
        torch.cuda.empty_cache()
        ws = sk.gram_workspace(Xt, Yt, scheme="approx", degree=DEGREE, compute="f32")
        ms = []
        for it in range(2):
            sk.sigkernel_gram(Xt, Yt, compute="f32", workspace=ws, out=G, **opts)
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            sk.sigkernel_backward(Wt, Xt, Yt, compute="f32", checkpoint=True, time_kernel=True, **opts)
            e1.record()
            e1.synchronize()
            if it >= 1:
                ms.append(e0.elapsed_time(e1))
        api["checkpoint_adjoint"] = {"backward_call_ms": statistics.mean(ms), "adjoint_kernel_ms": sk.last_kernel_ms(),
                                     "what": "sigkernel_backward with SK_FLAG_CHECKPOINT (no tape)"}
        line["api"] = api
        torch.cuda.empty_cache()

    if "fwd" in args.parts:  # forward only (the Gram alone)
        sf, kff, _, _ = run("f32", args.steps, 2, backward=False)
        kfo = statistics.mean(kff)
        line["forward_only"] = {"value": cells / (statistics.mean(sf) / 1e3), "unit": "cell-updates/s",
                                "ms_per_step": statistics.mean(sf),
                                "kernel": kernel_roofline("m_tc_kernel<16> + fwd_poly_kernel<float,6,6,false,1,false,"
                                                          "false,true> (no tape, M from the tensor cores)", kfo,
                                                          flops_per_cell(DEGREE, D) * cells, 0, p32)}

    if "f64" in args.parts:  # FP64 plain wavefront: forward, and fwd+bwd from an FP64 tape
        G64 = torch.empty_like(G)
        s64, k64, _, _ = run("f64", max(2, min(3, args.steps)), 1, backward=False, out=G64)
        k64avg = statistics.mean(k64)
        fb64, kf64, kb64, _ = run("f64", 2, 1, out=G64)
        sample_gram("f64", G64)
        line["fp64_plain_wavefront"] = {
            "forward": {"value": cells / (statistics.mean(s64) / 1e3), "unit": "cell-updates/s",
                        "ms_per_step": statistics.mean(s64),
                        "kernel": kernel_roofline("fwd_poly_kernel<double,6,6,false,1,false>", k64avg,
                                                  flops_per_cell(DEGREE, D) * cells, 0, p64)},
            "fwd_bwd": {"value": cells / (statistics.mean(fb64) / 1e3), "unit": "cell-updates/s",
                        "ms_per_step": statistics.mean(fb64), "tape_gb": round(tape_buf[0].numel() / 1e9, 2),
                        "forward_kernel": kernel_roofline("fwd_poly_kernel<double,6,6,false,1,false,true>",
                                                          statistics.mean(kf64),
                                                          tape_forward_flops_per_cell(DEGREE, D) * cells,
                                                          tape_forward_bytes(nx * nx, npts, esize=8), p64),
                        "adjoint_kernel": kernel_roofline("bwd_tape_kernel<double,6,false>", statistics.mean(kb64),
                                                          tape_adjoint_flops_per_cell(DEGREE) * cells,
                                                          tape_adjoint_bytes(nx * nx, npts, esize=8), p64)}}
        tape_buf[0] = None
        del G64
        torch.cuda.empty_cache()

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

    if "single" in args.parts:  # one pair of 33-point paths, d = 2, FP64: the plain method's latency
        Xs1 = W.brownian(2, 33, 2, seed=1 + 1000 * rank)
        Pa = torch.tensor(Xs1[:1], device=dev)
        Pb = torch.tensor(Xs1[1:], device=dev)
        i0 = torch.zeros(1, dtype=torch.int64, device=dev)
        o1 = torch.empty(1, dtype=torch.float64, device=dev)
        single = {"workload": "1 pair of 33-point Brownian paths, d=2, N(0,1/32) increments, FP64 (1,024 cells)"}
        gpu = {}
        for scheme, N, lam in (("approx", 4, 0), ("fd1", 2, 2), ("fd2", 2, 2)):
            f = lambda: sk.sigkernel_pairs(Pa, Pb, i0, i0, scheme=scheme, degree=N, dyadic=lam, compute="f64", out=o1)
            ms = timed_steps(f, 20, 3)
            key = f"{scheme}_N{N}_lam{lam}" if scheme == "approx" else f"{scheme}_lam{lam}"
            single[key] = {"us": ms * 1e3, "cell_updates_per_s": 1024 / (ms / 1e3)}
            samples[f"single_{key}"] = dict(xs=[Xs1[0]], ys=[Xs1[1]], pa=[0], pb=[0], scheme=scheme, N=N, lam=lam,
                                            gpu=o1.cpu().numpy().copy())
        # 64 linear pairs x = s u, y = t v against the closed form 0F1(;1;<u,v>) = sum_n <u,v>^n/(n!)^2
        Xl = W.linear(64, 33, 2, seed=2 + 1000 * rank)
        Yl = W.linear(64, 33, 2, seed=3 + 1000 * rank)
        il = torch.arange(64, dtype=torch.int64, device=dev)
        gl = sk.sigkernel_pairs(torch.tensor(Xl, device=dev), torch.tensor(Yl, device=dev), il, il, degree=12,
                                compute="f64").cpu().numpy()
        u, v = Xl[:, -1, :], Yl[:, -1, :]
        z = np.sum(u * v, axis=1)
        exact = np.array([sum(zi ** n / float(factorial(n)) ** 2 for n in range(60)) for zi in z])
        keep = np.abs(exact) >= 1e-3
        single["linear_pairs_closed_form"] = {
            "pairs": 64, "scheme": "approx N=12, FP64",
            "max_abs_err": float(np.max(np.abs(gl - exact))),
            "mape": float(np.mean(np.abs(gl - exact)[keep] / np.abs(exact[keep])))}
        line["single_pair"] = single

    if "gram_fd" in args.parts:  # the FD baseline on the same Gram beside the approximation scheme
        fd = {"workload": f"gram{nx}, FD1 at dyadic refinement 0/2/4 (sub-cells x1/16/256), FP32 and FP64"}
        Gf = torch.empty_like(G)
        for scheme, lam, comp in (("fd1", 0, "f32"), ("fd1", 2, "f32"), ("fd1", 4, "f32"), ("fd2", 2, "f32"),
                                  ("fd1", 0, "f64"), ("fd1", 2, "f64")):
            wsf = sk.gram_workspace(Xt, Yt, scheme=scheme, dyadic=lam, compute=comp)
            f = lambda: sk.sigkernel_gram(Xt, Yt, scheme=scheme, degree=2, dyadic=lam, compute=comp, workspace=wsf,
                                          out=Gf, sort=False)
            ms = timed_steps(f, 1 if lam == 4 else 3, 1)
            key = f"{scheme}_lam{lam}_{comp}"
            fd[key] = {"ms": ms, "cell_updates_per_s": cells / (ms / 1e3),
                       "sub_cell_updates_per_s": cells * 4 ** lam / (ms / 1e3)}
            sample_gram(f"gram_{key}", Gf, n=16, scheme=scheme, N=2, lam=lam)
        # gradients of the FD schemes: sigkernel_backward (forward recording per-column tapes in
        # chunks of pairs, the FD adjoint, the dk/dM contraction)
        for scheme, lam in (("fd1", 0), ("fd2", 2)):
            ms = timed_steps(lambda: sk.sigkernel_backward(Wt, Xt, Yt, scheme=scheme, degree=2, dyadic=lam,
                                                           compute="f32"), 2, 1)
            fd[f"{scheme}_lam{lam}_f32_fwd_bwd"] = {"ms": ms, "cell_updates_per_s": cells / (ms / 1e3),
                                                    "sub_cell_updates_per_s": cells * 4 ** lam / (ms / 1e3)}
        line["gram_fd"] = fd
        del Gf

    if "osc" in args.parts:  # 64 pairs of 1025-point oscillatory paths, d=4 (few long pairs: strip pipeline)
        Xo_np = W.oscillatory(64, 1025, 4, seed=5 + 1000 * rank)
        Yo_np = W.oscillatory(64, 1025, 4, seed=6 + 1000 * rank)
        Xo = torch.tensor(Xo_np, device=dev)
        Yo = torch.tensor(Yo_np, device=dev)
        io = torch.arange(64, dtype=torch.int64, device=dev)
        cells_o = 64 * 1024 * 1024
        osc = {"workload": "64 pairs, 1025 points on [0,1], d=4, sin(w t + phi) + N(0,1e-3), w ~ U(10,200)"}
        so = rng.choice(64, 4, replace=False)  # pairs the oracle checks
        for scheme, N, lam, comp in (("interp", 8, 0, "f32"), ("interp", 8, 0, "f64"), ("fd1", 2, 0, "f32"),
                                     ("fd1", 2, 2, "f32"), ("fd1", 2, 4, "f32"), ("fd1", 2, 6, "f32"),
                                     ("fd2", 2, 4, "f32"), ("fd_implicit", 2, 4, "f32")):
            o = torch.empty(64, dtype=torch.float64, device=dev)
            f = lambda: sk.sigkernel_pairs(Xo, Yo, io, io, scheme=scheme, degree=N, dyadic=lam, compute=comp, out=o)
            t = timed_steps(f, 1 if lam == 6 else 3, 1)
            key = f"{scheme}{N if scheme == 'interp' else ''}_lam{lam}_{comp}"
            osc[key] = {"ms": t, "cell_updates_per_s": cells_o / (t / 1e3),
                        "sub_cell_updates_per_s": cells_o * 4 ** lam / (t / 1e3)}
            if lam <= 4:
                oc = o.cpu().numpy()
                samples[f"osc_{key}"] = dict(xs=list(Xo_np), ys=list(Yo_np), pa=so, pb=so, scheme=scheme, N=N,
                                             lam=lam, gpu=oc[so])
        # gradients of the interpolation scheme (tape of cell inputs, one warp per pair: 64 warps)
        go = torch.ones(64, dtype=torch.float64, device=dev)
        t = timed_steps(lambda: sk.sigkernel_backward(go, Xo, Yo, io, io, scheme="interp", degree=8,
                                                      compute="f32"), 2, 1)
        osc["interp8_lam0_f32_fwd_bwd"] = {"ms": t, "cell_updates_per_s": cells_o / (t / 1e3),
                                           "note": "sigkernel_backward: forward recording the tape of cell inputs "
                                                   "(one warp per pair), the adjoint, the contraction"}
        line["oscillatory"] = osc
        del Xo, Yo

    if "long" in args.parts:  # one pair of 16385-point paths, d=4: parallelism inside a single pair
        Xl_np = W.brownian(1, 16385, 4, seed=11 + 1000 * rank)
        Yl_np = W.brownian(1, 16385, 4, seed=12 + 1000 * rank)
        Xl = torch.tensor(Xl_np, device=dev)
        Yl = torch.tensor(Yl_np, device=dev)
        il = torch.zeros(1, dtype=torch.int64, device=dev)
        ol = torch.empty(1, dtype=torch.float64, device=dev)
        cells_l = 16384 * 16384
        t_grid = timed_steps(lambda: sk.sigkernel_pairs(Xl, Yl, il, il, compute="f32", out=ol), 2, 1)
        # the oracle checks a pair of 4097-point prefixes, swept the same way (a ring of 8 blocks)
        Xp, Yp = Xl[:, :4097].contiguous(), Yl[:, :4097].contiguous()
        op = sk.sigkernel_pairs(Xp, Yp, il, il, compute="f32").cpu().numpy()
        samples["long_prefix4097"] = dict(xs=[Xl_np[0, :4097]], ys=[Yl_np[0, :4097]], pa=[0], pb=[0],
                                          scheme="approx", N=DEGREE, lam=0, gpu=op)
        line["long_pair"] = {"workload": "1 pair of 16385-point Brownian paths, d=4, approx N=6, FP32: the pair's "
                                         "512 strips swept by a ring of 32 co-resident 16-warp blocks",
                             "cells": cells_l, "ms": t_grid, "cell_updates_per_s": cells_l / (t_grid / 1e3),
                             "oracle_check": "a pair of 4097-point prefixes in the same grid strip pipeline"}
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
        graph.replay()
        torch.cuda.synchronize()
        su = rng.choice(4096, 16, replace=False)
        samples["uneven"] = dict(xs=[W.round_bf16(Xs[k]) for k in su], ys=[W.round_bf16(Ys[k]) for k in su],
                                 pa=np.arange(16), pb=np.arange(16), scheme="approx", N=DEGREE, lam=0,
                                 gpu=ou.cpu().numpy()[su])
        line["uneven_batch"] = {
            "workload": "4096 pairs, lengths log-uniform in [64,4096], d=16, BF16 points, approx N=6, FP32 cells",
            "cells": cells_u, "autotuned_shape": shape, "ms": t_tuned,
            "cell_updates_per_s": cells_u / (t_tuned / 1e3), "graph_replay_ms": t_graph,
            "graph_cell_updates_per_s": cells_u / (t_graph / 1e3), "one_warp_per_pair_ms": t_one}
        sk.autotune_clear()
        del PX, PY, graph

    if "mmd" in args.parts:  # MMD^2 fwd+bwd: 256 + 256 paths, 513 points, d=32, FP32
        nm = args.mmd_n
        Am_np = W.brownian(nm, 513, 32, seed=7 + 1000 * rank)
        Bm_np = W.brownian(nm, 513, 32, seed=8 + 1000 * rank, drift=0.5, vol=1.2)
        Am = torch.tensor(Am_np, device=dev)
        Bm = torch.tensor(Bm_np, device=dev)
        cells_m = (nm * (nm + 1) // 2 * 2 + nm * nm) * 512 * 512
        t_f = timed_steps(lambda: sk.sigkernel_mmd2(Am, Bm, degree=6, compute="f32"), 2, 1)
    if "mmd" in args.parts and args.mmd_forward_only:
        line["mmd2_forward_only"] = {"workload": f"{nm} + {nm} paths, 513 points, d=32, approx N=6, FP32",
                                     "cells": cells_m, "forward_ms": t_f}
        del Am, Bm
    elif "mmd" in args.parts:
        t_fb = timed_steps(lambda: sk.sigkernel_mmd2(Am, Bm, degree=6, compute="f32", grads=True), 2, 1)
        # the same with every contraction on the FMA pipe (tiled M forward, FMA dk/dM contraction)
        t_f0 = timed_steps(lambda: sk.sigkernel_mmd2(Am, Bm, degree=6, compute="f32", tensor_cores=False), 1, 1)
        t_fb0 = timed_steps(lambda: sk.sigkernel_mmd2(Am, Bm, degree=6, compute="f32", grads=True,
                                                      tensor_cores=False), 1, 1)
        labels = sk.split_labels(1000, nm, nm, seed=9 + rank)
        ws_t = sk.mmd2_test_workspace(Am, Bm, 1000, compute="f32")
        out_t = torch.empty(1002, dtype=torch.float64, device=dev)
        t_test = timed_steps(lambda: sk.sigkernel_mmd2_test(Am, Bm, labels=labels, compute="f32", workspace=ws_t,
                                                            out=out_t), 2, 1)
        # Gram entries of the three blocks, with the options sigkernel_mmd2 uses, for the oracle check
        sa_, sb_ = rng.integers(0, nm, 16), rng.integers(0, nm, 16)
        for name, P1, P2, n1, n2 in (("AB", Am, Bm, Am_np, Bm_np), ("AA", Am, Am, Am_np, Am_np),
                                     ("BB", Bm, Bm, Bm_np, Bm_np)):
            gm = sk.sigkernel_pairs(P1, P2, torch.tensor(sa_, device=dev), torch.tensor(sb_, device=dev),
                                    degree=6, compute="f32").cpu().numpy()
            samples[f"mmd_K{name}"] = dict(xs=list(n1), ys=list(n2), pa=sa_, pb=sb_, scheme="approx", N=6, lam=0,
                                           gpu=gm)
        line["mmd2"] = {"workload": f"{nm} + {nm} paths, 513 points, d=32 (Brownian vs drift 0.5, vol 1.2), approx "
                                    "N=6, FP32, symmetric K_AA/K_BB + K_AB; M_ij from a tcgen05 GEMM per chunk of "
                                    "pairs (three BF16 parts, FP32 accumulation); gradients from forward tapes in "
                                    "chunks of pairs (tape <= 64 GiB per chunk), dk/dM contracted on the tensor cores",
                        "cells": cells_m, "forward_ms": t_f, "fwd_bwd_ms": t_fb,
                        "forward_cell_updates_per_s": cells_m / (t_f / 1e3),
                        "fwd_bwd_cell_updates_per_s": cells_m / (t_fb / 1e3),
                        "fma_pipe_only": {"forward_ms": t_f0, "fwd_bwd_ms": t_fb0,
                                          "note": "SK_FLAG_NO_TC: tiled M on the FMA pipe, FMA dk/dM contraction"},
                        "permutation_test_1000_ms": t_test,
                        "permutation_test_p_value": out_t[1].item(),
                        "oracle_check": "16 sampled entries of each Gram block through sigkernel_pairs"}
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
            line["cpu_baseline"], line["mape_vs_fp64_oracle"] = cpu_baseline(X, Y, samples)
        print(json.dumps(line))
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
