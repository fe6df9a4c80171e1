#!/usr/bin/env python
"""Benchmark of the parallel Kalman filter + RTS smoother on GB300.

Metric: smoothed steps/s (steps of a sequence whose filtering and smoothing
posteriors have all been computed), one step of the benchmark = one full pass
of the hot path (filtering elements built from y, forward scan, smoothing
elements built from the filtered moments, reverse scan) over one sequence.

Workload (default): 2-D Wiener-velocity tracking model, nx = 4, ny = 2,
dt = 0.1, q = 1, R = I, m0 = 0, P0 = I, T = 2^20 steps, synthetic data
simulated from the model with a fixed seed (one independent sequence per
rank under torchrun: weak scaling, no collective on the data path).

    python bench.py [--steps K] [--warmup W] [--T T]
    python bench.py --impl reference      # the FP64 CPU oracle, same metric

Prints one JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402

METRIC = "smoothed steps/s"
UNIT = "steps/s"
FP32_LANES_PER_SM = 128
NUM_SMS = 152
SM_MAX_MHZ = 2070.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--T", type=int, default=1 << 20)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true",
                    help="default workload: leave out the batched measurement beside the headline")
    ap.add_argument("--workload", default="long", choices=["long", "batched", "precision", "serving", "tv", "hmm"],
                    help="long: one T=2^20 nx=4 sequence per GPU (default); batched: 4096 sequences, "
                         "lengths log-uniform in [256, 16384], nx in {2,4,6}; precision: nx=32 T=65536; "
                         "serving: Poisson request streams, nx in {4,8}, T log-uniform in [64, 2^18]; "
                         "tv: one T=2^20 nx=4 sequence with a time-varying model (irregular sampling); "
                         "hmm: one T=2^20 discrete-state sequence, K=8 regimes")
    ap.add_argument("--batch", type=int, default=4096)
    ap.add_argument("--hmm-k", type=int, default=8, choices=[2, 4, 8, 16, 32], help="hmm: number of states")
    ap.add_argument("--rates", default="100,300,1000,3000,10000", help="serving: request rates (req/s)")
    ap.add_argument("--duration", type=float, default=10.0, help="serving: seconds of arrivals per rate")
    ap.add_argument("--streams", type=int, default=3, help="serving: launches in flight")
    ap.add_argument("--budget-gb", type=float, default=80.0, help="serving: device-memory admission budget")
    return ap.parse_args()


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ---------------------------------------------------------------- work model
def bytes_per_step(nx: int, ny: int) -> dict:
    """Algorithmic DRAM bytes per step of each kernel (FP32), fused path:
    the forward scan reads y and writes the filtered mean + covariance; the
    reverse scan reads those and writes the smoothed ones."""
    post = 4 * (nx + nx * nx)
    return {"filter": 4 * ny + post, "smoother": 2 * post}


def flops_per_step(N: int, M: int, fused_smoothing: bool = True, block_fold: bool = None) -> dict:
    """Floating-point operations per step of each kernel's per-step work
    (FMA = 2).  The forward scan folds one measurement element into its block
    aggregate, applies it to the running filtered posterior, and -- fused into
    the same pass -- builds the step's Lemma 5 smoothing element from that
    posterior and folds it into the block's smoothing aggregate (Lemma 6).
    The fold is the linear block fold of a time-invariant model at nx <= 6
    (the innovation and two N x M products per step; `block_fold`), else the
    rank-M form of Lemma 4.  The reverse scan rebuilds the Lemma 5 element and
    applies it to the running smoothed posterior.  Block-level scan, look-back
    and per-model coefficient work are not counted."""
    if block_fold is None:
        block_fold = fused_smoothing
    s = N * (N + 1) // 2
    sm = M * (M + 1) // 2
    chol = M * M * M // 3 + 3 * M
    meas = 2 * (N * M + sm) + M
    fold = 2 * (3 * N * N * M + M * N * N + 2 * N * sm + sm * N + 2 * N ** 3 + s * N + 2 * s * M
                + N * N + 3 * N * M + sm) + chol
    adv = 2 * (N * N * M + sm * N + 2 * N * sm + 3 * N * M + N * N + s * M + N ** 3 + s * N) + chol
    sel = 2 * (N ** 3 + s * N + N ** 3 // 6 + N * N * (N - 1) + 2 * N * N + s * N) + 2 * N * N + N
    scomb = 2 * (N ** 3 + s * N + N * N + N ** 3)
    sadv = 2 * (N ** 3 + N * N + s * N)
    lbf = M + 2 * (2 * N * M)
    if fused_smoothing:
        first = lbf if block_fold else fold + meas
        return {"filter": first + adv + meas + sel + scomb, "smoother": sel + sadv}
    # warp-per-chain kernels (nx >= 8): the reverse scan folds its own blocks
    return {"filter": fold + adv + 2 * meas, "smoother": 2 * sel + scomb + sadv}


def tv_bytes_per_step(nx: int, ny: int) -> dict:
    """Algorithmic DRAM bytes per step of the time-varying path (FP32, u = d =
    0 so not read).  Element kernel: reads y_k, F_k, Q_k, H_k, R_k and writes
    the Lemma 3 element in measurement form (A, C lower, U, b, w).  Forward
    scan: reads that element and the next step's F, Q (for the fused Lemma 5
    element), writes the filtered mean + covariance.  Reverse scan: reads
    those moments and the next step's F, Q, writes the smoothed moments."""
    s = nx * (nx + 1) // 2
    model = 4 * (2 * nx * nx + ny * nx + ny * ny)
    elem = 4 * (nx * nx + s + ny * nx + nx + ny)
    post = 4 * (nx + nx * nx)
    trans = 4 * 2 * nx * nx
    return {"elements": 4 * ny + model + elem, "filter": elem + trans + post,
            "smoother": post + trans + post}


def tensor_flops_per_step(N: int, M: int) -> dict:
    """Algorithmic (FP32-equivalent, FMA = 2) flops per step of the dense
    products the nx >= 32 kernels run on the tensor cores.  Forward scan: the
    block fold of a measurement element (3 N^3 and 6 N^2 M products) and its
    application to the running posterior (2 N^3, 4 N^2 M).  Reverse scan:
    the Lemma 5 element (4 N^3), its block fold (3 N^3) and its application
    (2 N^3).  The pivoted inverses (CUDA cores) and the tile-level combines are
    not counted."""
    return {"filter": 2 * (5 * N ** 3 + 10 * N * N * M), "smoother": 2 * 9 * N ** 3}


def tf32_peak():
    """Dense TF32 tensor peak of this GPU: the measured bf16 GEMM peak times
    the nominal TF32 / bf16 ratio (1.1 / 2.25 PFLOP/s)."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["bf16_tflops"]) * 1.1 / 2.25, "measured bf16 GEMM x nominal TF32/bf16 (1.1/2.25)"
    return 1900.0 * 1.1 / 2.25, "fallback bf16 1.9 PFLOP/s x nominal TF32/bf16 (1.1/2.25)"


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1].split()[0]))
                smax.append(float(parts[2].split()[0]))
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- CPU oracle
def output_errors(got, ref) -> dict:
    """Errors of the GPU outputs (fmean, fcov, smean, scov as float arrays)
    against the oracle's FP64 ones, max over steps: normwise relative
    (|dm|_inf / max(|m|_inf, max_i sqrt(P_ii)); |dP|_max / |P|_max), the
    means' error in posterior standard deviations, |dm|_2 / sqrt(lambda_min(P)),
    and the largest use of the bound 0.01 sd + 24 ulps of the value (an FP32
    output cannot resolve less than its own ulp; at T = 2^20 one ulp of the
    position is several posterior sd)."""
    out = {}
    for name, g, r, P in (("fmean", got[0], ref[0], ref[1]), ("smean", got[2], ref[2], ref[3])):
        g = np.asarray(g, dtype=np.float64)
        d = g - r
        sd_scale = np.sqrt(np.abs(np.diagonal(P, axis1=-2, axis2=-1))).max(-1)
        rel = np.abs(d).max(-1) / np.maximum(np.abs(r).max(-1), sd_scale)
        s = np.sqrt(np.maximum(np.linalg.eigvalsh(P)[..., 0], np.finfo(np.float64).tiny))
        e = np.linalg.norm(d, axis=-1) / s
        ulp = np.linalg.norm(np.spacing(np.abs(r).astype(np.float32)).astype(np.float64), axis=-1) / s
        out[name] = {"rel": float(rel.max()), "sd": float(e.max()),
                     "sd_bound_use": float((e / (0.01 + 24.0 * ulp)).max())}
    for name, g, r in (("fcov", got[1], ref[1]), ("scov", got[3], ref[3])):
        d = np.abs(np.asarray(g, dtype=np.float64) - r).max((-2, -1)) / np.abs(r).max((-2, -1))
        out[name] = {"rel": float(d.max())}
    return out


def cpu_oracle_rate(seq, seconds: float, gpu_out=None) -> dict:
    """The FP64 oracle (sequential KF + RTS, one core) on the same sequence,
    repeated until `seconds` of CPU work have run (at least once).  With the
    GPU's outputs for this sequence, the first pass's results also give the
    line's `max_err`."""
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    reps = 0
    first = None
    while True:
        r = oracle.kf_rts(seq.model, seq.y)
        if first is None:
            first = r
        reps += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    res = {"value": reps * seq.T / el, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"{reps} full passes over the T={seq.T} sequence ({el:.1f} s, 1 thread)"}
    if gpu_out is not None:
        res["_max_err"] = output_errors(gpu_out, first)
    return res


# The sources that define each recorded kernel's code (its traffic record is
# dropped when any of them changes).
KERNEL_SOURCES = {
    "filter_scan_kernel": ["ks_ops.cuh", "ks_async.cuh", "ks_scan.cuh", "ks_impl.cuh", "ks_inst_4_2.cu"],
    "smoother_scan_kernel": ["ks_ops.cuh", "ks_async.cuh", "ks_scan.cuh", "ks_impl.cuh", "ks_inst_4_2.cu"],
    "tfilter_reduce+spine+apply": ["ks_tc.cuh", "ks_tscan.cuh"],
    "tsmoother_reduce+spine+apply": ["ks_tc.cuh", "ks_tscan.cuh"],
    "tv:elements": ["ks_ops.cuh", "ks_scan.cuh", "ks_impl.cuh"],
    "hmm:filter": ["ks_scan.cuh", "ks_hmm.cuh", "ks_hmm.cu"],
    "hmm:smoother": ["ks_scan.cuh", "ks_hmm.cuh", "ks_hmm.cu"],
    "tv:filter": ["ks_ops.cuh", "ks_async.cuh", "ks_scan.cuh", "ks_impl.cuh", "ks_inst_4_2.cu"],
    "tv:smoother": ["ks_ops.cuh", "ks_async.cuh", "ks_scan.cuh", "ks_impl.cuh", "ks_inst_4_2.cu"],
    "mixed_filter_kernel": ["ks_ops.cuh", "ks_async.cuh", "ks_scan.cuh", "ks_impl.cuh", "ks_mixed.cuh",
                            "ks_mixed32.cu"],
}


def source_hash(kernel: str) -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1905_13002_gb300", "csrc")
    for f in sorted(KERNEL_SOURCES.get(kernel, os.listdir(csrc))):
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(f.encode() + fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel: str, T: int):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel sources and holds the figure for this sequence
    length (another T runs another chunk variant); else None."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    e = d.get(kernel)
    if not e or e.get("source_hash") != source_hash(kernel) or e.get("T") != T:
        return None
    return e.get("dram_bytes_per_launch_full")


# ---------------------------------------------------------------- reference arm
def run_reference(args, rank, world):
    if rank != 0:
        return
    seq = workloads.tracking_sequence(args.T, seed=workloads.SEED_BASE + 2)
    import oracle
    oracle.build()
    # Each step: a bounded sample of the workload (a prefix of the sequence
    # sized so that W + K steps take about a minute or less).
    Ts = min(args.T, 1 << 18)
    sub = workloads.Sequence(seq.model, seq.y[:Ts])
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.kf_rts(sub.model, sub.y)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
    ms = 1e3 * statistics.mean(times)
    value = Ts / (ms / 1e3)
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": "wiener_velocity_2d nx=4 ny=2 dt=0.1 q=1 R=I", "T": args.T,
                      "T_sample_per_step": Ts},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                            "sample": f"first {Ts} steps of the T={args.T} sequence per step"},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


# ---------------------------------------------------------------- our arm
def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.workload == "batched":
        run_batched(args, rank, world, local)
        return
    if args.workload == "serving":
        run_serving(args, rank, world, local)
        return
    if args.workload == "hmm":
        run_hmm(args, rank, world, local)
        return
    run_single(args, rank, world, local, mode=args.workload)


def block_length(ks, nx: int, T: int) -> dict:
    """Steps per thread the library uses for this call, whether full blocks
    go through the linear block fold, and where the rule came from (the
    tuner's cache for this device, or the built-in table)."""
    from paper_1905_13002_gb300 import tune
    src = os.path.relpath(tune.APPLIED, ROOT) if tune.APPLIED else "built-in table"
    return {"steps_per_thread": ks.chunk_steps(nx, T) if nx <= 6 else None,
            "block_fold": bool(ks.chunk_fold(nx, T)) if nx <= 6 else False, "rules": src}


def launches_per_call(nx: int, T: int) -> int:
    """Kernels one ks_smooth call launches: nx <= 6: preparation, forward scan,
    its refinement retry (returns at once unless needed), reverse scan;
    nx = 32: preparation, then per scan a reduce, one spine launch per
    Kogge-Stone level over the tiles of 3 chains x 72 steps, and an apply."""
    if nx <= 6:
        return 4
    tiles = -(-T // (3 * 72))
    levels = (tiles - 1).bit_length() if tiles > 1 else 0
    return 1 + 2 * (2 + levels)


def run_single(args, rank, world, local, mode):
    import torch
    import torch.distributed as dist

    import paper_1905_13002_gb300 as ks
    from paper_1905_13002_gb300 import _build

    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    if local == 0:
        _build.build()
    if world > 1:
        dist.barrier()
    precision, tv = mode == "precision", mode == "tv"
    if precision:
        T = 65536 if args.T == (1 << 20) else args.T
        seq = workloads.config_precision(T=T)
        if rank:
            rng = np.random.default_rng(np.random.PCG64(workloads.SEED_BASE + 4 + rank))
            _, y = workloads.simulate(seq.model, T, rng)
            seq = workloads.Sequence(seq.model, y)
        wl = "random_stable nx=32 ny=8 F=O diag(U[0.9,0.99]) Q=0.1I H~N(0,1/32) R=0.5I"
    elif tv:
        T = args.T
        seq = workloads.irregular_tracking(T, seed=workloads.SEED_BASE + 6 + rank)
        wl = ("irregular_tracking_2d nx=4 ny=2 time-varying: dt_k~logU[0.02,0.5] (F_k, Q_k), "
              "R_k=r_k I r_k~logU[0.25,4], q=1 u=d=0 m0=0 P0=I")
    else:
        T = args.T
        seq = workloads.tracking_sequence(T, seed=workloads.SEED_BASE + 2 + rank)
        wl = "wiener_velocity_2d nx=4 ny=2 dt=0.1 q=1 R=I m0=0 P0=I"
    dev = torch.device("cuda", local)
    m = seq.model
    nx, ny = m.nx, m.ny
    if tv:   # u = d = 0: passed as absent
        model = ks.Model.create(m.F, m.Q, m.H, m.R, m.m0, m.P0, device=dev)
    else:
        model = ks.Model.create(m.F, m.Q, m.H, m.R, m.m0, m.P0, u=m.u, d=m.d, device=dev)
    y = torch.as_tensor(seq.y, dtype=torch.float32, device=dev)
    ws = ks.alloc_workspace(model, T, ks.KS_WS_ELEMENTS)
    fm = torch.empty(T, nx, device=dev)
    fP = torch.empty(T, nx, nx, device=dev)
    sm = torch.empty(T, nx, device=dev)
    sP = torch.empty(T, nx, nx, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # > 129 MB L2
    stream = torch.cuda.current_stream()

    def step(events=None):
        ks.smooth(model, y, ws, fmean=fm, fcov=fP, smean=sm, scov=sP, events=events)

    for _ in range(max(args.warmup, 3)):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    if ks.status(ws) != ks.KS_OK:
        raise SystemExit("device status not OK after warm-up")

    # one call captured in a CUDA graph (as a serving loop would run it),
    # timed with events around each replay
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        step()
    graph.replay()
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    clocks = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    tot = []
    for i in range(args.steps):
        flush.zero_()                       # L2 flushed between timed steps, outside the events
        ev[0].record()
        graph.replay()
        ev[3].record()
        ev[3].synchronize()
        tot.append(ev[0].elapsed_time(ev[3]))
    # per-kernel times: the same call launched directly, with events between
    # the preparation, the forward scan (and its retry) and the reverse scan
    kel, kf, ksm = [], [], []
    for i in range(args.steps):
        flush.zero_()
        step(ev)
        ev[3].synchronize()
        kel.append(ev[0].elapsed_time(ev[1]))
        kf.append(ev[1].elapsed_time(ev[2]))
        ksm.append(ev[2].elapsed_time(ev[3]))
    torch.cuda.synchronize()
    time.sleep(0.3)
    clk = clocks.stop()
    if world > 1:
        dist.barrier()
    st = ks.status(ws)
    if st != ks.KS_OK:
        raise SystemExit(f"device status {st} after the timed steps")
    lat = {"p50_ms": float(np.percentile(tot, 50)), "p99_ms": float(np.percentile(tot, 99))}
    ms = statistics.mean(tot)
    if world > 1:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    value = T * world / (ms / 1e3)

    # ---- end to end through the public API with host buffers: every step
    # copies its measurements in from pinned host memory, runs ks_smooth and
    # reads its smoothed means and covariances back.  Consecutive steps
    # alternate between two streams (each with its own device buffers and
    # workspace), so one step's copies overlap the next step's kernels: the
    # figure is K steps over the wall time of all K.
    y_h = torch.as_tensor(seq.y, dtype=torch.float32).pin_memory()
    # a time-varying model is part of each call's input: its per-step arrays
    # are copied in with y
    model_h = {k: getattr(model, k).cpu().pin_memory() for k in ("F", "Q", "H", "R")} if tv else {}
    lanes = []
    for j in range(2):
        mj = model if j == 0 else (ks.Model.create(m.F, m.Q, m.H, m.R, m.m0, m.P0, device=dev) if tv else model)
        lanes.append({"stream": torch.cuda.Stream(device=dev), "model": mj, "y": torch.empty_like(y),
                      "ws": ws if j == 0 else ks.alloc_workspace(model, T, ks.KS_WS_ELEMENTS),
                      "sm": sm if j == 0 else torch.empty(T, nx, device=dev),
                      "sP": sP if j == 0 else torch.empty(T, nx, nx, device=dev),
                      "sm_h": torch.empty(T, nx, dtype=torch.float32).pin_memory(),
                      "sP_h": torch.empty(T, nx, nx, dtype=torch.float32).pin_memory()})

    def e2e_call(L):
        with torch.cuda.stream(L["stream"]):
            for k, h in model_h.items():
                getattr(L["model"], k).copy_(h, non_blocking=True)
            L["y"].copy_(y_h, non_blocking=True)
            ks.smooth(L["model"], L["y"], L["ws"], smean=L["sm"], scov=L["sP"], keep_filtered=False)
            L["sm_h"].copy_(L["sm"], non_blocking=True)
            L["sP_h"].copy_(L["sP"], non_blocking=True)

    main_s = torch.cuda.current_stream()
    for i in range(args.warmup):
        e2e_call(lanes[i % 2])
    torch.cuda.synchronize()
    flush.zero_()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(main_s)
    for L in lanes:
        L["stream"].wait_stream(main_s)
    for i in range(args.steps):
        e2e_call(lanes[i % 2])
    for L in lanes:
        main_s.wait_stream(L["stream"])
    b.record(main_s)
    b.synchronize()
    e2e_ms = a.elapsed_time(b) / args.steps
    for L in lanes:
        if ks.status(L["ws"]) != ks.KS_OK:
            raise SystemExit("device status not OK after the end-to-end steps")
    e2e = {"value": T * world / (e2e_ms / 1e3), "unit": UNIT,
           "h2d_bytes_per_step": int(y_h.numel() * 4 + sum(h.numel() * 4 for h in model_h.values())),
           "d2h_bytes_per_step": int((lanes[0]["sm_h"].numel() + lanes[0]["sP_h"].numel()) * 4),
           "how": "consecutive calls alternate between 2 streams (copies of one overlap the kernels of the next)"}
    del lanes

    # ---- roofline of the dominant kernel
    hbm, which = peaks()
    if tv:
        roof = tv_roofline(nx, ny, T, hbm, which, {"elements": statistics.mean(kel), "filter": statistics.mean(kf),
                                                   "smoother": statistics.mean(ksm)})
    bps = bytes_per_step(nx, ny)
    fps = flops_per_step(nx, ny, fused_smoothing=nx <= 6,
                         block_fold=nx <= 6 and not tv and ks.chunk_fold(nx, T) == 1)
    kernels = {"filter": statistics.mean(kf), "smoother": statistics.mean(ksm)}
    if not tv:
        roof = scan_roofline(nx, ny, T, hbm, which, kernels, bps, fps)
        roof["prep_ms"] = round(statistics.mean(kel), 4)   # model constants (and block-fold coefficients)

    # the batched workload beside it (the metric's "batched FP32 scan vs plain
    # scan"): one mixed-size launch per scan, and the plain per-sequence scan
    # the outputs of the last timed call, for the error against the oracle
    want_err = world == 1 and not args.no_cpu_baseline
    host_out = tuple(t.cpu().numpy() for t in (fm, fP, sm, sP)) if want_err else None
    batched = None
    if mode == "long" and not args.no_batched:
        del fm, fP, sm, sP, ws, flush
        batched = measure_batched(args, rank, world, dev, full=False)
        batched["roofline"]["traffic"] = recorded_traffic("mixed_filter_kernel", batched["config"]["total_steps"])
        batched.pop("_seqs", None)
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": wl, "T": T,
                      "sequences_per_gpu": 1, "parallelism": f"replicas{world}",
                      "launch": "one ks_smooth call replayed as a CUDA graph (kernel times: direct calls)",
                      "block_length": block_length(ks, nx, T),
                      "l2": "flushed between timed steps (256 MiB memset outside the events)"},
           "clocks": {k: clk[k] for k in ("sm_mhz", "sm_max_mhz", "reasons")},
           "gpu_launches": 2 * launches_per_call(nx, T) * args.steps, "latency": lat, "e2e": e2e, "roofline": roof}
    if world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_oracle_rate(seq, args.cpu_seconds, host_out)
        out["max_err"] = out["cpu_baseline"].pop("_max_err")
    if batched is not None:
        out["batched"] = batched
    print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


def tv_roofline(nx, ny, T, hbm, which, kernels):
    """Time-varying path: every kernel is HBM-side (the element kernel
    streams the per-step model; the scans stream elements and posteriors)."""
    bps = tv_bytes_per_step(nx, ny)
    dom = max(kernels, key=kernels.get)
    gbs = bps[dom] * T / (kernels[dom] / 1e3) / 1e9
    names = {"elements": "tv_elements_kernel", "filter": "filter_scan_kernel (materialised elements)",
             "smoother": "smoother_scan_kernel (time-varying)"}
    return {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
            "traffic": recorded_traffic("tv:" + dom, T), "kernel": names[dom], "peak_source": which,
            "ms_per_launch": kernels[dom], "bytes_per_step": bps,
            "kernels_ms": {k: round(v, 4) for k, v in kernels.items()},
            "gbs_by_kernel": {k: round(bps[k] * T / (v / 1e3) / 1e9, 1) for k, v in kernels.items()}}


def scan_roofline(nx, ny, T, hbm, which, kernels, bps, fps):
    """Time-invariant scans: the dominant kernel against the ALU, HBM or
    tensor roof, whichever its work model reaches first."""
    dom = max(kernels, key=kernels.get)
    dur_s = kernels[dom] / 1e3
    gbs = bps[dom] * T / dur_s / 1e9
    alu_peak = NUM_SMS * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
    tfl = fps[dom] * T / dur_s / 1e12
    kname = ({"filter": "filter_scan_kernel", "smoother": "smoother_scan_kernel"} if nx <= 6 else
             {"filter": "tfilter_reduce+spine+apply", "smoother": "tsmoother_reduce+spine+apply"} if nx >= 32 else
             {"filter": "gfilter_reduce+spine+apply", "smoother": "gsmoother_reduce+spine+apply"})[dom]
    traffic = recorded_traffic(kname, T)
    if nx >= 32:
        tpeak, tsrc = tf32_peak()
        tfs = tensor_flops_per_step(nx, ny)[dom]
        ttf = tfs * T / dur_s / 1e12
        roof = {"bound": "tensor", "achieved": ttf, "peak": tpeak, "unit": "TFLOP/s", "frac": ttf / tpeak,
                "traffic": traffic, "kernel": kname, "peak_source": tsrc, "ms_per_launch": kernels[dom],
                "split": "3xTF32: 3 TF32 mma per FP32 product, so the tensor pipe issues 3x achieved",
                "tensor_flops_per_step": tfs, "hbm_frac": gbs / hbm, "bytes_per_step": bps[dom],
                "kernels_ms": {k: round(v, 4) for k, v in kernels.items()}}
    elif tfl / alu_peak >= gbs / hbm:
        roof = {"bound": "alu", "achieved": tfl, "peak": alu_peak, "unit": "TFLOP/s",
                "frac": tfl / alu_peak, "traffic": traffic}
    else:
        roof = {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s",
                "frac": gbs / hbm, "traffic": traffic}
    if nx < 32:
        roof.update({"kernel": kname, "peak_source": which if roof["bound"] == "hbm" else
                     "152 SMs x 128 FP32 lanes x 2 x 2070 MHz",
                     "ms_per_launch": kernels[dom], "hbm_frac": gbs / hbm, "alu_frac": tfl / alu_peak,
                     "bytes_per_step": bps[dom], "flops_per_step": fps[dom],
                     "kernels_ms": {k: round(v, 4) for k, v in kernels.items()}})

    return roof


# ---------------------------------------------------------------- discrete-state workload
def hmm_work_per_step(K: int) -> tuple[dict, dict]:
    """(flops, algorithmic DRAM bytes) per step of the two HMM scans (FP32,
    FMA = 2).  Forward: the fold of the step element ((f Pi) then the
    likelihood scaling and row normalisation), its application to the running
    marginal, the step's Definition 2 element from that marginal and its fold
    into the thread's smoothing aggregate; reads lik, writes filt and loglik.
    Reverse: the Definition 2 element and its application; reads filt, writes
    smooth.  Tile-level combines are not counted."""
    fold = 2 * K ** 3 + 3 * K * K + 2 * K
    adv = 2 * K * K + 3 * K
    sel = 2 * K * K + K
    smul = 2 * K ** 3
    flops = {"filter": fold + adv + sel + smul, "smoother": sel + 2 * K * K}
    nbytes = {"filter": 4 * K + 4 * K + 4, "smoother": 4 * K + 4 * K}
    return flops, nbytes


def run_hmm(args, rank, world, local):
    import torch
    import torch.distributed as dist

    import paper_1905_13002_gb300 as ks
    from paper_1905_13002_gb300 import _build

    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    if local == 0:
        _build.build()
    if world > 1:
        dist.barrier()
    K = args.hmm_k
    T = args.T
    seq = workloads.hmm_sequence(K, T, seed=workloads.SEED_BASE + 7 + rank)
    dev = torch.device("cuda", local)
    model = ks.HmmModel.create(seq.pi, seq.Pi, device=dev)
    lik = torch.as_tensor(seq.lik, dtype=torch.float32, device=dev)
    ws = torch.empty(ks.hmm_workspace_bytes(K, T), dtype=torch.uint8, device=dev)
    ks.lib().ks_workspace_init(ks._p(ws), ws.numel(), ks._stream(None))
    filt = torch.empty(T, K, device=dev)
    smooth = torch.empty(T, K, device=dev)
    ll = torch.empty(T, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def step(events=None):
        ks.hmm_smooth(model, lik, ws, filt=filt, smooth=smooth, loglik=ll, events=events)

    for _ in range(max(args.warmup, 3)):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    if ks.status(ws) != ks.KS_OK:
        raise SystemExit("device status not OK after warm-up")
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    clocks = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    for i in range(args.steps):
        flush.zero_()
        step(evs[i])
    torch.cuda.synchronize()
    time.sleep(0.3)
    clk = clocks.stop()
    if world > 1:
        dist.barrier()
    if ks.status(ws) != ks.KS_OK:
        raise SystemExit("device status not OK after the timed steps")
    tot = [e[0].elapsed_time(e[3]) for e in evs]
    kf = statistics.mean(e[1].elapsed_time(e[2]) for e in evs)
    ksm = statistics.mean(e[2].elapsed_time(e[3]) for e in evs)
    ms = statistics.mean(tot)
    if world > 1:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    value = T * world / (ms / 1e3)

    # end to end: likelihoods in from pinned host memory, marginals and
    # log-likelihoods back
    lik_h = torch.as_tensor(seq.lik, dtype=torch.float32).pin_memory()
    filt_h = torch.empty(T, K).pin_memory()
    smooth_h = torch.empty(T, K).pin_memory()
    ll_h = torch.empty(T).pin_memory()
    lik_d = torch.empty_like(lik)
    e2e_times = []
    for i in range(args.warmup + args.steps):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        lik_d.copy_(lik_h, non_blocking=True)
        ks.hmm_smooth(model, lik_d, ws, filt=filt, smooth=smooth, loglik=ll)
        filt_h.copy_(filt, non_blocking=True)
        smooth_h.copy_(smooth, non_blocking=True)
        ll_h.copy_(ll, non_blocking=True)
        b.record()
        b.synchronize()
        if i >= args.warmup:
            e2e_times.append(a.elapsed_time(b))
    e2e = {"value": T * world / (statistics.mean(e2e_times) / 1e3), "unit": UNIT,
           "h2d_bytes_per_step": int(lik_h.numel() * 4),
           "d2h_bytes_per_step": int((filt_h.numel() + smooth_h.numel() + ll_h.numel()) * 4)}

    flops, nbytes = hmm_work_per_step(K)
    if K <= 8:
        launches_per_step = 3
    else:   # prep, then per scan a reduce, ceil(log2(tiles)) spine levels and an apply
        tiles = -(-T // (64 * 128 // K))    # 64 steps per chain, 128 / K chains per tile
        launches_per_step = 1 + 2 * (2 + max(0, math.ceil(math.log2(tiles))))
    kernels = {"filter": kf, "smoother": ksm}
    dom = max(kernels, key=kernels.get)
    dur_s = kernels[dom] / 1e3
    alu_peak = NUM_SMS * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
    tfl = flops[dom] * T / dur_s / 1e12
    hbm, which = peaks()
    gbs = nbytes[dom] * T / dur_s / 1e9
    roof = ({"bound": "alu", "achieved": tfl, "peak": alu_peak, "unit": "TFLOP/s", "frac": tfl / alu_peak}
            if tfl / alu_peak >= gbs / hbm else
            {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm})
    roof.update({"traffic": recorded_traffic("hmm:" + dom, T) if K == 8 else None,
                 "kernel": f"hmm_{dom}_kernel<{K}>" if K <= 8 else f"hmmw {dom} reduce+spine+apply (K={K})",
                 "peak_source": "152 SMs x 128 FP32 lanes x 2 x 2070 MHz" if roof["bound"] == "alu" else which,
                 "ms_per_launch": kernels[dom], "alu_frac": tfl / alu_peak, "hbm_frac": gbs / hbm,
                 "flops_per_step": flops[dom], "bytes_per_step": nbytes[dom],
                 "kernels_ms": {k: round(v, 4) for k, v in kernels.items()}})
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": f"regime-switching HMM K={K}, stay 0.95, y~N(x, 0.6^2), Gaussian likelihood rows",
                      "T": T, "sequences_per_gpu": 1, "parallelism": f"replicas{world}",
                      "l2": "flushed between timed steps (256 MiB memset outside the events)"},
           "clocks": {k: clk[k] for k in ("sm_mhz", "sm_max_mhz", "reasons")},
           "gpu_launches": launches_per_step * args.steps, "latency": {"p50_ms": float(np.percentile(tot, 50)),
                                                       "p99_ms": float(np.percentile(tot, 99))},
           "e2e": e2e, "roofline": roof}
    if world == 1 and not args.no_cpu_baseline:
        from oracle import hmm as ohmm
        Ts = min(T, 1 << 16)
        t0 = time.perf_counter()
        reps = 0
        while True:
            ohmm.forward_backward(seq.pi, seq.Pi, seq.lik[:Ts])
            reps += 1
            el = time.perf_counter() - t0
            if el >= args.cpu_seconds:
                break
        out["cpu_baseline"] = {"value": reps * Ts / el, "unit": UNIT, "cores": 1, "kind": "oracle",
                               "sample": f"{reps} passes over the first {Ts} steps ({el:.1f} s, 1 thread, numpy)"}
    print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


# ---------------------------------------------------------------- batched workload
def cpu_oracle_batched(seqs, seconds: float) -> dict:
    """The FP64 oracle over the batch's sequences on all host cores (one
    sequence per task; the C oracle releases the GIL), on a bounded sample:
    sequences in order until `seconds` have elapsed."""
    from concurrent.futures import ThreadPoolExecutor
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    done_steps = 0
    done = 0
    with ThreadPoolExecutor(max_workers=cores) as ex:
        i = 0
        while i < len(seqs) and time.perf_counter() - t0 < seconds:
            chunk = seqs[i:i + 4 * cores]
            list(ex.map(lambda q: oracle.kf_rts(q.model, q.y), chunk))
            done_steps += sum(q.T for q in chunk)
            done += len(chunk)
            i += len(chunk)
    el = time.perf_counter() - t0
    return {"value": done_steps / el, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"first {done} of {len(seqs)} sequences ({done_steps} steps, {el:.1f} s, {cores} threads)"}


def measure_batched(args, rank, world, dev, full: bool) -> dict:
    """The batched workload (4096 sequences, log-uniform lengths, nx in {2, 4,
    6}) through ks_smooth_batched: one preparation, one forward and one
    reverse launch over all three state sizes, captured in a CUDA graph.
    Returns the JSON fields of the measurement; `full` adds the end-to-end
    figure and the per-size comparison (three ks_smooth_batch calls on three
    streams), which the default benchmark line leaves out."""
    import torch
    import torch.distributed as dist

    import paper_1905_13002_gb300 as ks

    seqs = workloads.config_batched(B=args.batch, seed=workloads.SEED_BASE + 3 + rank)
    total = sum(q.T for q in seqs)
    groups = []
    for nx in (6, 4, 2):
        g = [q for q in seqs if q.model.nx == nx]
        if not g:
            continue
        batch = ks.ModelBatch.create([q.model for q in g], [q.T for q in g], device=dev)
        y = torch.as_tensor(np.concatenate([q.y for q in g]), dtype=torch.float32, device=dev)
        T = int(y.shape[0])
        outs = (torch.empty(T, nx, device=dev), torch.empty(T, nx, nx, device=dev),
                torch.empty(T, nx, device=dev), torch.empty(T, nx, nx, device=dev))
        groups.append({"nx": nx, "B": batch.B, "T": T, "batch": batch, "y": y, "outs": outs})
    sizes = [(g["nx"], g["nx"] // 2, g["B"], g["T"]) for g in groups]
    ws = torch.zeros(ks.workspace_bytes_batched(sizes), dtype=torch.uint8, device=dev)
    pairs = [(g["batch"], g["y"]) for g in groups]
    outs = [g["outs"] for g in groups]

    def step():
        ks.smooth_batched(pairs, ws, outs=outs)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    if ks.status(ws) != ks.KS_OK:
        raise SystemExit("batched: device status not OK after warm-up")
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        step()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def timed(fn, n):
        out = []
        for _ in range(n):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            b.synchronize()
            out.append(a.elapsed_time(b))
        return out

    timed(graph.replay, 2)
    clocks = ClockSampler(dev.index or 0)
    if world > 1:
        dist.barrier()
    clocks.start()
    time.sleep(0.3)
    times = timed(graph.replay, args.steps)
    time.sleep(0.3)
    clk = clocks.stop()
    if world > 1:
        dist.barrier()
    if ks.status(ws) != ks.KS_OK:
        raise SystemExit("batched: device status not OK after timing")
    ms = statistics.mean(times)
    if world > 1:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    res = {"value": total * world / (ms / 1e3), "unit": UNIT, "ms_per_step": ms,
           "latency": {"p50_ms": float(np.percentile(times, 50)), "p99_ms": float(np.percentile(times, 99))},
           "clocks": {k: clk[k] for k in ("sm_mhz", "sm_max_mhz", "reasons")},
           "gpu_launches": 4 * args.steps,
           "config": {"workload": "batched: log-uniform T in [256,16384], nx in {2,4,6} Wiener-velocity, "
                                  "q~U[0.5,2], R=rI r~U[0.1,1]", "sequences": len(seqs), "total_steps": total,
                      "groups": [{"nx": g["nx"], "B": g["B"], "T": g["T"]} for g in groups],
                      "launch": "ks_smooth_batched: prep + forward + refinement retry + reverse launches over "
                                "all sizes (CUDA graph)",
                      "block_length": block_length(ks, 0, total),
                      "l2": "flushed between timed steps (256 MiB memset outside the events)"}}

    # the plain single-sequence scan, one ks_smooth call per sequence, same GPU
    plain = []
    for q in seqs:
        m = q.model
        model = ks.Model.create(m.F, m.Q, m.H, m.R, m.m0, m.P0, device=dev)
        yq = torch.as_tensor(q.y, dtype=torch.float32, device=dev)
        wsq = ks.alloc_workspace(model, q.T)
        o = [torch.empty(q.T, m.nx, device=dev), torch.empty(q.T, m.nx, m.nx, device=dev),
             torch.empty(q.T, m.nx, device=dev), torch.empty(q.T, m.nx, m.nx, device=dev)]
        plain.append((model, yq, wsq, o))

    def plain_pass():
        for model, yq, wsq, o in plain:
            ks.smooth(model, yq, wsq, fmean=o[0], fcov=o[1], smean=o[2], scov=o[3])

    plain_pass()
    torch.cuda.synchronize()
    pms = statistics.median(timed(plain_pass, 3))
    res["plain_scan"] = {"value": total / (pms / 1e3), "unit": UNIT, "ms_per_pass": pms,
                         "how": "ks_smooth once per sequence, sequentially on one stream"}
    del plain

    # roofline over the whole step: algorithmic bytes and flops of all groups
    hbm, which = peaks()
    nbytes = nflops = 0
    for g in groups:
        bps = bytes_per_step(g["nx"], g["nx"] // 2)
        fps = flops_per_step(g["nx"], g["nx"] // 2, block_fold=ks.chunk_fold(0, total) == 1)
        nbytes += (bps["filter"] + bps["smoother"]) * g["T"]
        nflops += (fps["filter"] + fps["smoother"]) * g["T"]
    dur = ms / 1e3
    gbs = nbytes / dur / 1e9
    tfl = nflops / dur / 1e12
    alu_peak = NUM_SMS * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
    if tfl / alu_peak >= gbs / hbm:
        roof = {"bound": "alu", "achieved": tfl, "peak": alu_peak, "unit": "TFLOP/s", "frac": tfl / alu_peak}
    else:
        roof = {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm}
    roof.update({"traffic": None, "kernel": "whole step (mixed prep + forward + reverse launches)",
                 "hbm_frac": gbs / hbm, "alu_frac": tfl / alu_peak,
                 "peak_source": "152 SMs x 128 FP32 lanes x 2 x 2070 MHz" if roof["bound"] == "alu" else which})
    res["roofline"] = roof
    if not full:
        return res

    # the same groups as three per-size segmented calls on three streams (the
    # form before the mixed-size launch), for comparison
    per = []
    for g in groups:
        wsg = torch.zeros(ks.workspace_bytes_batch(g["nx"], g["nx"] // 2, g["B"], g["T"]), dtype=torch.uint8,
                          device=dev)
        per.append((g, wsg, torch.cuda.Stream(device=dev)))

    def per_size():
        main = torch.cuda.current_stream()
        for g, wsg, s in per:
            s.wait_stream(main)
            with torch.cuda.stream(s):
                fm, fP, sm, sP = g["outs"]
                ks.smooth_batch(g["batch"], g["y"], wsg, fmean=fm, fcov=fP, smean=sm, scov=sP)
        for _, _, s in per:
            main.wait_stream(s)

    for _ in range(3):
        per_size()
    g2 = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g2):
        per_size()
    per_ms = statistics.mean(timed(g2.replay, args.steps))
    res["per_size_calls"] = {"value": total / (per_ms / 1e3), "unit": UNIT, "ms_per_step": per_ms,
                             "how": "3 ks_smooth_batch calls (one per nx) on 3 streams, one CUDA graph"}

    # end to end through the public API: each group's measurements in from
    # pinned host memory, its smoothed means and covariances back
    hosts = []
    for g in groups:
        nx = g["nx"]
        hosts.append((g["y"].cpu().pin_memory(), torch.empty(g["T"], nx).pin_memory(),
                      torch.empty(g["T"], nx, nx).pin_memory(), torch.empty_like(g["y"])))
    e2e_pairs = [(g["batch"], h[3]) for g, h in zip(groups, hosts)]

    def e2e_step():
        for h in hosts:
            h[3].copy_(h[0], non_blocking=True)
        ks.smooth_batched(e2e_pairs, ws, outs=outs)
        for g, h in zip(groups, hosts):
            h[1].copy_(g["outs"][2], non_blocking=True)
            h[2].copy_(g["outs"][3], non_blocking=True)

    e2e_times = timed(e2e_step, args.warmup + args.steps)[args.warmup:]
    if ks.status(ws) != ks.KS_OK:
        raise SystemExit("batched: device status not OK after the end-to-end steps")
    res["e2e"] = {"value": total * world / (statistics.mean(e2e_times) / 1e3), "unit": UNIT,
                  "h2d_bytes_per_step": int(sum(h[0].numel() * 4 for h in hosts)),
                  "d2h_bytes_per_step": int(sum((h[1].numel() + h[2].numel()) * 4 for h in hosts))}
    res["_seqs"] = seqs
    return res


def run_batched(args, rank, world, local):
    import torch
    import torch.distributed as dist

    from paper_1905_13002_gb300 import _build

    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if local == 0:
        _build.build()
    if world > 1:
        dist.barrier()
    res = measure_batched(args, rank, world, dev, full=True)
    seqs = res.pop("_seqs")
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    out = {"metric": METRIC, "value": res["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": res["ms_per_step"], "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic"}
    out.update({k: v for k, v in res.items() if k not in ("value", "unit", "ms_per_step")})
    if world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_oracle_batched(seqs, args.cpu_seconds)
    print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


def run_serving(args, rank, world, local):
    """Open-loop Poisson request streams through the continuous-batching
    server, one stream per rate; each rank serves its own stream (replicas)."""
    import torch
    import torch.distributed as dist

    from paper_1905_13002_gb300 import _build, serving

    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    if local == 0:
        _build.build()
    if world > 1:
        dist.barrier()
    models = workloads.serving_models(seed=workloads.SEED_BASE + 5)
    ys = workloads.serving_measurements(models, 1 << 18, seed=workloads.SEED_BASE + 5 + 100 * rank)
    pinned = {nx: [torch.from_numpy(y).pin_memory() for y in v] for nx, v in ys.items()}
    sets = {(nx, nx // 2): serving.ModelSet(models[nx]) for nx in models}
    budget = int(args.budget_gb * 1e9)
    rates = [float(r) for r in args.rates.split(",")]

    def requests(rate, n, seed):
        arr = workloads.serving_arrivals(rate, n, seed)
        return [serving.Request(i, a.nx, a.nx // 2, a.T, a.model, pinned[a.nx][a.model][:a.T], a.t)
                for i, a in enumerate(arr)]

    serving.Server(serving.GpuLauncher(sets, streams=args.streams), budget, streams=args.streams).run(
        requests(rates[0], 64, workloads.SEED_BASE + 5 + 7919 + rank))          # warm-up
    clk = ClockSampler(local)
    clk.start()
    per_rate = {}
    launches = 0
    for rate in rates:
        n = max(1, int(round(rate * args.duration)))
        rs = requests(rate, n, workloads.SEED_BASE + 5 + 1000 * int(rate) + rank)
        gl = serving.GpuLauncher(sets, streams=args.streams)
        srv = serving.Server(gl, budget, streams=args.streams)
        done = srv.run(rs)
        launches += srv.stats.launches
        lg = gl.log
        dev_rate = {}
        for nx in sorted({e[0] for e in lg}):
            e = [x for x in lg if x[0] == nx]
            dev_rate[str(nx)] = sum(x[2] for x in e) / (sum(x[4] for x in e) / 1e3)
        lat = [r.latency * 1e3 for r in done]
        p = serving.percentiles(lat, (50, 99))
        steps = sum(r.T for r in done)
        span = max(r.done for r in done) - min(r.arrival for r in done)
        rate_steps = torch.tensor([steps / span], dtype=torch.float64, device="cuda")
        if world > 1:
            dist.all_reduce(rate_steps)
        per_rate[str(int(rate))] = {
            "requests": n, "steps": steps, "steps_per_s": float(rate_steps.item()),
            "offered_steps_per_s": rate * statistics.mean(r.T for r in rs) * world,
            "p50_ms": p[50], "p99_ms": p[99], "launches": srv.stats.launches,
            "mean_requests_per_launch": statistics.mean(srv.stats.batch_sizes),
            "max_reserved_gb": srv.stats.max_reserved / 1e9, "max_in_flight": srv.stats.max_in_flight,
            "launch_host_ms_mean": 1e3 * statistics.mean(x[3] for x in lg),
            "launch_device_ms_mean": statistics.mean(x[4] for x in lg),
            "device_steps_per_s_by_nx": dev_rate}
    clk_s = clk.stop()
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    top = per_rate[str(int(rates[-1]))]
    out = {"metric": METRIC, "value": top["steps_per_s"], "unit": UNIT, "n_gpus": world, "steps": len(rates),
           "warmup": 1, "ms_per_step": top["p50_ms"], "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": "serving: Poisson arrivals, T=round(exp(U[ln64, ln2^18])), nx in {4 (Wiener "
                                  "velocity, ny=2), 8 (random stable, ny=4)}, 16 models per nx",
                      "rates": rates, "seconds_per_rate": args.duration, "streams": args.streams,
                      "budget_gb": args.budget_gb, "parallelism": f"replicas{world}",
                      "value": "smoothed steps/s at the highest rate (completed steps / (last completion - "
                               "first arrival)); ms_per_step = its p50 latency",
                      "latency": "completion (CUDA event after the request's launch) - scheduled arrival"},
           "clocks": {k: clk_s[k] for k in ("sm_mhz", "sm_max_mhz", "reasons")},
           "gpu_launches": 4 * launches,   # a lower bound: nx = 8 calls also run spine launches
           "latency": {"p50_ms": top["p50_ms"], "p99_ms": top["p99_ms"]},
           "rates": per_rate}
    if world == 1 and not args.no_cpu_baseline:
        sample = requests(rates[-1], 400, workloads.SEED_BASE + 5 + 31)
        seqs = [workloads.Sequence(models[r.nx][r.model], ys[r.nx][r.model][:r.T].astype(np.float64))
                for r in sample]
        out["cpu_baseline"] = cpu_oracle_batched(seqs, args.cpu_seconds)
    print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
