#!/usr/bin/env python3
"""Benchmark of the double FFT filter (arXiv:2305.01537, Sec. II.C) on GB300.

One step = one application of the whole filter (theta pass, then phi pass) to every field of the
28-field state of the Nr=128, Ntheta=64, Nphi=128 workload (29,360,128 points, FP64 in and out,
470 MB of I/O: larger than the 126 MB L2, so no flush is needed between steps).

Prints one JSON line. `value` is filtered points per second over all ranks (Gpoints/s) of the
plan's FP64 arithmetic (--precision selects another), timed on the device with CUDA events around
K steps after W warm-up steps, inputs already in HBM. `e2e` is the same metric through the
host-buffer C-ABI call (sph_filter_apply_host), with the host->device copy of the state and the
device->host copy of the result inside every step, next to the measured host-copy ceiling.
`variants` holds the other arithmetic forms (compensated FP32 pairs, the split-precision
tensor-core form) timed the same way on the same state, each with its largest per-field error
against the oracle on the oracle's sample of shells.

--impl reference times the oracle (the plain CPU definition) on the host cores instead.
Multi-GPU (torchrun): every rank filters its own copy of the state (independent shards, no
data collective: weak scaling); the slowest rank's time is reported.
"""
from __future__ import annotations

import argparse
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

from paper_2305_01537_gb300 import workloads as W  # noqa: E402

HBM_FALLBACK_GBS = 6800.0
# ALU roofs measured on this GPU model (GB300, 152 SMs) with an FMA-chain throughput probe: 8
# independent FMA chains per thread, 8 CTAs of 256 threads per SM, CUDA-event timing, the SM clock
# read from clock64 over the same kernel (1.8-2.06 GHz). FP64 FMA: 0.626 T/s (2.0-2.2 per SM per
# clock); FP32 FMA: 38.2 T/s; INT32 IMAD: 20.0 T/s (64 per SM per clock). tcgen05.mma kind::i8 is not
# available on sm_103a (ptxas rejects it), so no integer tensor-core rate exists.
FP64_FMA_PER_S = 0.626e12
FP32_FMA_PER_S = 38.2e12
FP64_PEAK_TFLOPS = 2 * FP64_FMA_PER_S / 1e12
FP64_PEAK_SOURCE = "measured FP64 FMA rate (FMA-chain probe on GB300): 0.626 T FMA/s x 2 flop"
# Compensated FP32 pairs: the measured FP32 FMA issue rate divided by the FP32 instructions one
# FP64-equivalent flop of the radix-8 butterfly costs (866 / 98 = 8.8)
DF_INSTR_PER_FLOP = 866.0 / 98.0
DF_PEAK_TFLOPS = FP32_FMA_PER_S / DF_INSTR_PER_FLOP / 1e12
DF_PEAK_SOURCE = ("FP64-equivalent rate of compensated FP32 pairs: measured FP32 FMA rate (38.2 T/s, FMA-chain "
                  "probe on GB300) / 8.8 FP32 instructions per FP64-equivalent flop of the radix-8 butterfly")


KERNEL_FAMILIES = {
    # CUDA sources whose device code each kernel family compiles from
    "plain": ["shell_kernel.cuh", "shell_inst.cu", "shell_dispatch.cu", "filter_plain.cu", "df32.h", "dfmath.h",
              "capi.cu"],  # capi.cu: which kernels an application launches (the split)
    "tc": ["tc.cu", "tc_plan.cu", "tc2_host.h"],
}


def kernel_sources_hash(family: str) -> str:
    """Hash of a kernel family's CUDA sources, to tell whether recorded ncu counters still describe
    the kernel."""
    import hashlib
    csrc = os.path.join(ROOT, "paper_2305_01537_gb300", "csrc")
    h = hashlib.sha256()
    for name in KERNEL_FAMILIES[family]:
        h.update(name.encode())
        with open(os.path.join(csrc, name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": HBM_FALLBACK_GBS, "bf16_tflops": 1900.0}, "fallback"


def algorithmic_flops(grid) -> float:
    """FFT-form flop count of one application: 5 log2(2 Ntheta) + 1 per point of a shell whose
    theta pass is active, 5 log2(Nphi) + 1 per point of an active ring. Identity shells (exponential
    or sharp filter with l_max >= Ntheta) and rings (m_max >= Nphi/2) cost nothing. Hybrid fields
    count as exponential ones: a lower bound, since the shells and rings where Jameson's detector
    fires (data dependent) are transformed too."""
    flops = 0.0
    th = (np.arange(grid.Ntheta) + 0.5) * math.pi / grid.Ntheta
    for v in range(grid.nvars):
        for i in range(grid.Nr):
            lm = max(grid.floor, 2 * grid.r[i] / grid.dr_min * grid.L[v])
            gauss = grid.kind[v] == W.GAUSS
            if gauss or lm < grid.Ntheta:
                flops += grid.Ntheta * grid.Nphi * (5 * math.log2(2 * grid.Ntheta) + 1)
            mm = np.maximum(grid.floor, 2 * grid.r[i] / grid.dr_min * np.sin(th) * grid.L[v])
            nact = grid.Ntheta if gauss else int((mm < grid.Nphi / 2).sum())
            flops += nact * grid.Nphi * (5 * math.log2(grid.Nphi) + 1)
    return flops


def tc_blocks(L: int):
    """The split-precision form's GEMM shapes for vectors of length L, as the plan builds them: levels
    while L/2^l is divisible by 4 with a quarter of at least 16 and a half of at least 32 (each level's
    two halves fill the 128 rows of one GEMM, K = N = the quarter padded to 16), then the base of length
    nb split into two halves of nb/2 (side by side in one GEMM with N = 2K when that needs no more than
    256 tensor-memory columns or the separate form's, else two GEMMs). Returns [(K, N, gemms)]."""
    pad = lambda n: (n + 15) // 16 * 16
    shapes, n = [], L
    while n % 4 == 0 and n // 4 >= 16 and n // 2 >= 32:
        shapes.append((pad(n // 4), pad(n // 4), 1))
        n //= 2
    kb = pad(n // 2)
    KA = max([kb] + [k for k, _, _ in shapes])
    NA = max([kb] + [nn for _, nn, _ in shapes])

    def cols(ka, na):
        c = 32
        while c < 3 * ka + 5 * na:
            c *= 2
        return c
    c_with = cols(KA, max(NA, 2 * kb))
    if c_with <= max(cols(KA, NA), 256) and c_with <= 512:
        shapes.append((kb, 2 * kb, 1))
    else:
        shapes.append((kb, kb, 2))
    return shapes


def tc_tile_flops(L: int, factored: bool) -> float:
    """Tensor-core flops of one tile of 64 vectors: every GEMM runs 128 rows (two per vector) for the
    21 digit pairs a + b <= 5, 2 flops per multiply-add; the factored form runs each block twice
    (forward to the modes and back)."""
    f = sum(g * 128.0 * K * N * 21 * 2 for K, N, g in tc_blocks(L))
    return 2 * f if factored else f


def tc_tensor_flops(grid) -> float:
    """Tensor-core flops of one application of the split-precision form: theta tiles of 64 doubled
    circles of the active shells (direct form, one GEMM per block, when Nphi/2 is a multiple of 64,
    else factored), phi tiles of 64 active rings (factored), with the activity rule of the FFT form."""
    th = (np.arange(grid.Ntheta) + 0.5) * math.pi / grid.Ntheta
    circles, rings = 0, 0
    for v in range(grid.nvars):
        for i in range(grid.Nr):
            lm = max(grid.floor, 2 * grid.r[i] / grid.dr_min * grid.L[v])
            gauss = grid.kind[v] == W.GAUSS
            if gauss or lm < grid.Ntheta:
                circles += grid.Nphi // 2
            mm = np.maximum(grid.floor, 2 * grid.r[i] / grid.dr_min * np.sin(th) * grid.L[v])
            rings += grid.Ntheta if gauss else int((mm < grid.Nphi / 2).sum())
    direct = (grid.Nphi // 2) % 64 == 0
    return (-(-circles // 64)) * tc_tile_flops(2 * grid.Ntheta, not direct) + (-(-rings // 64)) * tc_tile_flops(grid.Nphi, True)


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons every 200 ms while running."""

    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.window = None
        self._stop = threading.Event()
        self._proc = None

    def __enter__(self):
        try:
            self._proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except (OSError, FileNotFoundError):
            self._proc = None
            return self
        # nvidia-smi needs a moment before its first sample: wait for it (at most 3 s), so that a
        # short run still has samples to report
        t_end = time.time() + 3.0
        while not self.rows and time.time() < t_end and self._proc.poll() is None:
            time.sleep(0.02)
        return self

    def _read(self):
        for line in self._proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append((time.time(), parts[1:]))

    def mark(self, t0: float, t1: float):
        """Keep only the samples taken between wall-clock times t0 and t1 (the timed region)."""
        self.window = (t0, t1)

    def __exit__(self, *exc):
        if self._proc is not None:
            self._proc.terminate()
            try:
                self._proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self._proc.kill()

    def summary(self, window=None):
        """Median SM clock, max clock, throttle reasons and power over the samples taken inside
        `window` (wall-clock (t0, t1), default the marked one). When the window is shorter than the
        sampling interval and holds no sample, the whole run's samples (warm-up, timed regions and
        the end-to-end and variant runs around them) are reported instead, and `scope` says so."""
        window = window or self.window
        scope = "timed region"
        rows = [r for (t, r) in self.rows if window is None or window[0] <= t <= window[1] + 0.15]
        if not rows:
            rows = [r for (_, r) in self.rows]
            scope = "whole run (the timed region is shorter than the 100 ms sampling interval)"
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[4 + k].lower() == "active"})
        pw = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows), "scope": scope,
                "power_w_max": max(pw) if pw else None}


def combine_ranks(times_ms, units_per_rank: float, steps: int, device=None):
    """Max over ranks of each timed region (ms) and the whole-job rate of each: every rank
    processes `units_per_rank` units per step (independent shards, weak scaling), so the job's
    rate is world * units * steps / slowest time. Uses the default process group if initialised."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size() if dist.is_available() and dist.is_initialized() else 1
    t = torch.tensor([float(x) for x in times_ms], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    slow = [float(x) for x in t.cpu()]
    rates = [world * units_per_rank * steps / (ms * 1e-3) for ms in slow]
    return slow, rates


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def single_grid_workload(name):
    return {"state28_128x64x128": W.full_state_128x64x128, "state28_256x128x256": W.full_state_256x128x256,
            "state28_32x128x256": W.state_32x128x256, "hybrid28_128x64x128": W.hybrid_state_128x64x128,
            "hybrid28_256x128x256": W.hybrid_state_256x128x256, "hybrid28_32x128x256": W.hybrid_state_32x128x256}[name]()


def cpu_baseline(grid, x, seconds_target=10.0, stride0=16):
    """The oracle as it stands, on all host cores, over a stratified sample of shells (every s-th
    radial shell of every field), grown until it has run for about `seconds_target` seconds.
    Returns (record, radial indices of the sample, the oracle's output on the sample)."""
    import oracle
    threads = oracle.max_threads()
    stride = stride0
    total_pts, total_t = 0, 0.0
    sample_shells = 0
    while True:
        idx = np.arange(0, grid.Nr, stride)
        xs = np.ascontiguousarray(x[:, idx])
        t0 = time.perf_counter()
        ref = oracle.filter(xs, grid.parity, grid.kind, grid.L, grid.r[idx], grid.dr_min, grid.floor, eps=grid.eps)
        dt = time.perf_counter() - t0
        total_pts, total_t = xs.size, dt
        sample_shells = xs.shape[0] * xs.shape[1]
        if dt >= seconds_target / 4 or stride == 1:
            break
        stride = max(1, stride // 4)
    rec = {"value": total_pts / total_t / 1e9, "unit": "Gpoints/s", "cores": threads, "kind": "oracle",
           "sample": f"{sample_shells} shells (every {stride}th radial shell of all {grid.nvars} fields), "
                     f"{total_pts} points in {total_t:.2f} s"}
    return rec, idx, ref


def sample_error(y, idx, ref) -> float:
    """Largest per-field normalised max-norm error of the device result y (torch, [nvars][Nr][..])
    on the sampled radial shells idx against the oracle's output ref on them."""
    ys = y[:, idx].cpu().numpy()
    err = 0.0
    for v in range(ref.shape[0]):
        den = max(float(np.abs(ref[v]).max()), 1e-300)
        err = max(err, float(np.abs(ys[v] - ref[v]).max()) / den)
    return err


def run_reference(args):
    world, rank, _ = dist_setup()
    if rank != 0:
        return 0
    import oracle
    # the single-grid workloads run as named; the others fall back to the default state
    try:
        wl = single_grid_workload(args.workload)
    except KeyError:
        wl = W.full_state_128x64x128()
    g = wl.grids[0]
    x = wl.state()
    threads = oracle.max_threads()
    # each step: a bounded sample (every 16th radial shell of every field)
    idx = np.arange(0, g.Nr, 16)
    xs = np.ascontiguousarray(x[:, idx])
    for _ in range(args.warmup):
        oracle.filter(xs, g.parity, g.kind, g.L, g.r[idx], g.dr_min, g.floor, eps=g.eps)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.filter(xs, g.parity, g.kind, g.L, g.r[idx], g.dr_min, g.floor, eps=g.eps)
    dt = time.perf_counter() - t0
    value = xs.size * args.steps / dt / 1e9
    line = {
        "impl": "reference", "metric": "filtered Gpoints/s (theta+phi double FFT filter, FP64 I/O)",
        "value": value, "unit": "Gpoints/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl.name, "Nr": g.Nr, "Ntheta": g.Ntheta, "Nphi": g.Nphi, "nvars": g.nvars,
                   "sample_per_step": f"{xs.shape[1]} of {g.Nr} radial shells x {g.nvars} fields"},
        "cpu_baseline": {"value": value, "unit": "Gpoints/s", "cores": threads, "kind": "oracle",
                         "sample": f"{xs.shape[0] * xs.shape[1]} shells per step ({xs.size} points)"},
        "e2e": {"value": value, "unit": "Gpoints/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def _timed(fn, steps, warmup, stream):
    """Run fn warmup times, then time `steps` calls with CUDA events on `stream` (ms total)."""
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def run_batch(args):
    """Six uneven grids (28 fields each) filtered three times per step (one filter per RK3 substep),
    replayed as one CUDA graph per step. Tensor-core plans run all six grids in one persistent launch
    per application; the plain forms' plans are autotuned and run one launch set per grid."""
    import torch
    from paper_2305_01537_gb300 import Batch, Plan, SPH_PREC_F64, SPH_PREC_F32X2, SPH_PREC_SPLIT_TC
    prec = {"f64": SPH_PREC_F64, "f32x2": SPH_PREC_F32X2, "tc": SPH_PREC_SPLIT_TC}[args.precision]
    wl = W.batched_six_grids()
    xs, outs, plans = [], [], []
    for n, g in enumerate(wl.grids):
        xs.append(torch.from_numpy(wl.state(n)).cuda())
        outs.append(torch.empty_like(xs[-1]))
        plans.append(Plan.from_grid(g, precision=prec))
        if prec != SPH_PREC_SPLIT_TC:
            plans[-1].autotune(xs[-1], outs[-1])
    b = Batch(plans)
    stream = torch.cuda.current_stream()
    captured0 = sum(p.launch_count for p in plans)
    b.capture(xs, outs, 3, stream)
    per_graph = sum(p.launch_count for p in plans) - captured0
    with ClockSampler(0) as clk:
        t0 = time.time()
        ms = _timed(lambda: b.launch(stream), args.steps, args.warmup, stream)
        clk.mark(t0, time.time())
    points = wl.points * 3
    value = points * args.steps / (ms * 1e-3) / 1e9
    peaks, src = measured_peaks()
    gbs = 16.0 * points * args.steps / (ms * 1e-3) / 1e9
    print(json.dumps({
        "metric": "filtered Gpoints/s (theta+phi double FFT filter, FP64 I/O)", "value": value, "unit": "Gpoints/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": DTYPE_NAME[args.precision],
        "data": "synthetic",
        "config": {"workload": wl.name, "grids": [[g.Nr, g.Ntheta, g.Nphi, g.nvars] for g in wl.grids],
                   "applications_per_step": 3, "precision": args.precision,
                   "launch": ("one CUDA graph per step: one persistent launch per application over all six grids"
                              if prec == SPH_PREC_SPLIT_TC else
                              "one CUDA graph per step (per-grid kernels on parallel branches)")},
        "hbm": {"achieved_gbs": gbs, "peak_gbs": peaks["hbm_gbs"], "frac": gbs / peaks["hbm_gbs"], "peak_source": src},
        "gpu_launches": args.steps * per_graph, "launches_per_application": per_graph / 3,
        "clocks": clk.summary()}), flush=True)
    return 0


def run_chain(args):
    """loss = sum w (F o tanh o ... o F x)^2 over 8 filters on the 8-field 128x64x128 state; one step
    is the forward chain and its gradient (8 fused adjoint launches)."""
    import torch
    from paper_2305_01537_gb300 import Plan, SPH_PREC_F64, SPH_PREC_F32X2
    from paper_2305_01537_gb300.autograd import chain_loss
    prec = SPH_PREC_F32X2 if args.precision == "f32x2" else SPH_PREC_F64
    wl = W.chain_8field()
    g = wl.grids[0]
    x = torch.from_numpy(wl.state() * 0.1).cuda()
    w = torch.from_numpy(W.chain_weights(g)).cuda()
    plan = Plan.from_grid(g, precision=prec)
    stream = torch.cuda.current_stream()

    def step():
        xd = x.detach().requires_grad_(True)
        chain_loss(xd, plan, w, 8).backward()

    with ClockSampler(0) as clk:
        t0 = time.time()
        n0 = plan.launch_count
        ms = _timed(step, args.steps, args.warmup, stream)
        per_step = (plan.launch_count - n0) // (args.steps + args.warmup)
        clk.mark(t0, time.time())
    points = g.points * 16  # 8 forward + 8 adjoint filter applications
    value = points * args.steps / (ms * 1e-3) / 1e9
    print(json.dumps({
        "metric": "filtered Gpoints/s (theta+phi double FFT filter, FP64 I/O)", "value": value, "unit": "Gpoints/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
        "config": {"workload": wl.name, "filters": 8, "step": "forward chain + backward", "precision": args.precision},
        "gpu_launches": args.steps * per_step, "clocks": clk.summary()}), flush=True)
    return 0


def run_constraints(args):
    """The algebraic-constraint map after filtering (Sec. II.C) on a 13-field state (h 11..33, A
    11..33, lapse) of 256 x 64 x 128 points (218 MB, larger than L2), in place; the theta-filtered
    shells are those with l_max < Ntheta for the metric fields' filter (exponential, L = 3)."""
    import numpy as np
    import torch
    from paper_2305_01537_gb300 import enforce_constraints
    Nr, Nth, Nph = 256, 64, 128
    rng = np.random.default_rng(21)
    x = rng.standard_normal((13, Nr, Nth, Nph))
    x[:6] *= 0.05
    x[12] = rng.uniform(0.0, 1.0, (Nr, Nth, Nph))
    r = np.arange(Nr) + 0.5
    flags = (np.maximum(2.0, 2.0 * r * 3.0) < Nth).astype(np.uint8)
    hv, av, al = list(range(6)), list(range(6, 12)), 12
    x_host = torch.from_numpy(x).pin_memory()
    xd = x_host.cuda()
    fd = torch.from_numpy(flags).cuda()
    stream = torch.cuda.current_stream()
    points = Nr * Nth * Nph
    bh = flags.astype(bool)[:, None, None] & (x[12] < 0.3)
    n_bh = int(bh.sum())
    # algorithmic bytes: standard points read 13 and write 12 values, modified ones read 7 and write 1
    bytes_per_step = 8.0 * ((points - n_bh) * 25 + n_bh * 8)
    with ClockSampler(0) as clk:
        t0 = time.time()
        ms = _timed(lambda: enforce_constraints(xd, hv, av, al, fd, 0.3, stream), args.steps, args.warmup, stream)
        clk.mark(t0, time.time())
    out_host = torch.empty_like(x_host).pin_memory()

    def e2e_step():
        xd.copy_(x_host, non_blocking=True)
        enforce_constraints(xd, hv, av, al, fd, 0.3, stream)
        out_host.copy_(xd, non_blocking=True)

    e2e_ms = _timed(e2e_step, args.steps, args.warmup, stream)
    peaks, src = measured_peaks()
    gbs = bytes_per_step * args.steps / (ms * 1e-3) / 1e9
    print(json.dumps({
        "metric": "constraint-map Gpoints/s (Sec. II.C algebraic constraints after filtering, FP64)",
        "value": points * args.steps / (ms * 1e-3) / 1e9, "unit": "Gpoints/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "constraints_256x64x128", "Nr": Nr, "Ntheta": Nth, "Nphi": Nph, "fields": 13,
                   "modified_form_points": n_bh, "l2": f"state ({8 * 13 * points / 1e6:.0f} MB) larger than L2; no flush"},
        "roofline": {"bound": "hbm", "achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                     "frac": gbs / peaks["hbm_gbs"], "traffic": None, "peak_source": src,
                     "kernel": "constraint_kernel", "bytes_per_launch": bytes_per_step},
        "e2e": {"value": points * args.steps / (e2e_ms * 1e-3) / 1e9, "unit": "Gpoints/s",
                "h2d_bytes_per_step": 8 * 13 * points, "d2h_bytes_per_step": 8 * 13 * points},
        "gpu_launches": args.steps, "clocks": clk.summary()}), flush=True)
    return 0


PRECISIONS = ("f64", "f32x2", "tc", "spectral")
DTYPE_NAME = {"f64": "f64", "f32x2": "f32x2", "tc": "bf16x_split", "spectral": "f64"}


def roofline_for(precision, g, avg_kernel_s, points, peaks, src, traffic, label):
    """Roofline object of one application: the FP64 pipe for the FP64 form, the FP32 instruction rate
    (through the compensated arithmetic's FP32 instructions per flop) for the FP32-pair form, the bf16
    tensor pipe for the split-precision form."""
    flops = algorithmic_flops(g)
    tflops = flops / avg_kernel_s / 1e12
    if precision in ("f64", "spectral"):
        return {"bound": "alu", "achieved": tflops, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": tflops / FP64_PEAK_TFLOPS, "traffic": traffic, "peak_source": FP64_PEAK_SOURCE,
                "kernel": label, "flops_per_launch": flops}
    if precision == "f32x2":
        return {"bound": "alu", "achieved": tflops, "peak": DF_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": tflops / DF_PEAK_TFLOPS, "traffic": traffic, "peak_source": DF_PEAK_SOURCE,
                "kernel": label, "flops_per_launch": flops}
    tc_flops = tc_tensor_flops(g)
    tc_tflops = tc_flops / avg_kernel_s / 1e12
    peak = peaks["bf16_tflops"]
    return {"bound": "tensor", "achieved": tc_tflops, "peak": peak, "unit": "TFLOP/s", "frac": tc_tflops / peak,
            "traffic": traffic, "peak_source": f"bf16_tflops (burst) of {src}", "kernel": label,
            "flops_per_launch": tc_flops}


def time_plan(plan, x, y, steps, warmup, stream):
    """W untimed applications, then K timed ones with one event pair per application on the
    launching stream. Returns (total ms, per-application ms list, kernel launches in the timed
    region)."""
    import torch
    for _ in range(warmup):
        plan.apply(x, out=y)
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    launched0 = plan.launch_count
    t_start.record(stream)
    for k in range(steps):
        evs[k][0].record(stream)
        plan.apply(x, out=y)
        evs[k][1].record(stream)
    t_end.record(stream)
    torch.cuda.synchronize()
    return t_start.elapsed_time(t_end), [a.elapsed_time(b) for a, b in evs], plan.launch_count - launched0


def host_copy_ceiling(x_host, stream_a, stream_b, reps=3):
    """Measured host<->device copy rates for the state's bytes (pinned host memory): host to device
    alone, device to host alone, and both directions at once on two streams (the bound of an
    end-to-end step that moves the state in and the result out). GB/s, best of `reps`."""
    import torch
    dev = torch.empty_like(x_host, device="cuda")
    dev2 = torch.empty_like(x_host, device="cuda")
    back = torch.empty_like(x_host).pin_memory()
    nbytes = x_host.numel() * x_host.element_size()

    def best(fn):
        ms = []
        for _ in range(reps + 1):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream_a)
            fn()
            stream_a.wait_stream(stream_b)
            e1.record(stream_a)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        return min(ms[1:])

    def h2d():
        with torch.cuda.stream(stream_a):
            dev.copy_(x_host, non_blocking=True)

    def d2h():
        with torch.cuda.stream(stream_a):
            back.copy_(dev2, non_blocking=True)

    def both():
        stream_b.wait_stream(stream_a)
        with torch.cuda.stream(stream_a):
            dev.copy_(x_host, non_blocking=True)
        with torch.cuda.stream(stream_b):
            back.copy_(dev2, non_blocking=True)

    t_h2d, t_d2h, t_both = best(h2d), best(d2h), best(both)
    return {"bytes_each_way": nbytes, "h2d_gbs": nbytes / t_h2d / 1e6, "d2h_gbs": nbytes / t_d2h / 1e6,
            "both_ways_ms": t_both, "both_ways_gbs_each": nbytes / t_both / 1e6}


def measure_workload(wl_name, precisions, steps, warmup, sample_stride):
    """One single-grid workload at several precisions (same state, out of place): Gpoints/s, ms per
    application, kernel launches, and the largest per-field error against the oracle on the shells of
    every `sample_stride`-th radius (the oracle's own output on those shells)."""
    import torch
    import oracle
    from paper_2305_01537_gb300 import Plan, SPH_PREC_F64, SPH_PREC_F32X2, SPH_PREC_SPLIT_TC
    code = {"f64": SPH_PREC_F64, "f32x2": SPH_PREC_F32X2, "tc": SPH_PREC_SPLIT_TC}
    wl = single_grid_workload(wl_name)
    g = wl.grids[0]
    xh = wl.state()
    idx = np.arange(0, g.Nr, sample_stride)
    t0 = time.perf_counter()
    ref = oracle.filter(np.ascontiguousarray(xh[:, idx]), g.parity, g.kind, g.L, g.r[idx], g.dr_min, g.floor, eps=g.eps)
    oracle_s = time.perf_counter() - t0
    x = torch.from_numpy(xh).cuda()
    del xh
    y = torch.empty_like(x)
    stream = torch.cuda.current_stream()
    out = {}
    for p in precisions:
        plan = Plan.from_grid(g, precision=code[p])
        ms, kms, launched = time_plan(plan, x, y, steps, warmup, stream)
        assert plan.sync_status() == 0
        out[p] = {"value": g.points * steps / (ms * 1e-3) / 1e9, "unit": "Gpoints/s", "ms_per_step": ms / steps,
                  "dtype": DTYPE_NAME[p], "gpu_launches_per_application": launched / steps,
                  "max_err_vs_oracle": sample_error(y, idx, ref),
                  "hbm_frac": 16.0 * g.points / (statistics.mean(kms) * 1e-3) / 1e9 / measured_peaks()[0]["hbm_gbs"]}
        del plan
    del x, y
    torch.cuda.empty_cache()
    return {"workload": wl.name, "Nr": g.Nr, "Ntheta": g.Ntheta, "Nphi": g.Nphi, "nvars": g.nvars,
            "points": g.points, "steps": steps, "warmup": warmup,
            "err_sample": f"every {sample_stride}th radius of all {g.nvars} fields ({len(idx) * g.nvars} shells; "
                          f"oracle {oracle_s:.1f} s)",
            "by_precision": out}


def measure_batch(steps, warmup):
    """The six uneven grids, three applications per step as one CUDA graph per step, tensor-core plans
    (one persistent launch per application over all grids)."""
    import torch
    from paper_2305_01537_gb300 import Batch, Plan, SPH_PREC_SPLIT_TC
    wl = W.batched_six_grids()
    xs, outs, plans = [], [], []
    for n, g in enumerate(wl.grids):
        xs.append(torch.from_numpy(wl.state(n)).cuda())
        outs.append(torch.empty_like(xs[-1]))
        plans.append(Plan.from_grid(g, precision=SPH_PREC_SPLIT_TC))
    b = Batch(plans)
    stream = torch.cuda.current_stream()
    c0 = sum(p.launch_count for p in plans)
    b.capture(xs, outs, 3, stream)
    per_graph = sum(p.launch_count for p in plans) - c0
    ms = _timed(lambda: b.launch(stream), steps, warmup, stream)
    ok = all(p.sync_status() == 0 for p in plans)
    points = wl.points * 3
    res = {"workload": wl.name, "grids": [[g.Nr, g.Ntheta, g.Nphi, g.nvars] for g in wl.grids], "precision": "tc",
           "value": points * steps / (ms * 1e-3) / 1e9, "unit": "Gpoints/s", "ms_per_step": ms / steps,
           "applications_per_step": 3, "gpu_launches_per_application": per_graph / 3, "status_ok": ok,
           "steps": steps, "warmup": warmup,
           "launch": "one CUDA graph per step; one persistent launch per application over all six grids"}
    del b, plans, xs, outs
    torch.cuda.empty_cache()
    return res


def measure_chain(precision, steps, warmup):
    """loss = sum w (F o tanh o ... o F x)^2 over 8 filters on the 8-field 128x64x128 state; one step is
    the forward chain and its gradient (8 + 8 fused launches)."""
    import torch
    from paper_2305_01537_gb300 import Plan, SPH_PREC_F64, SPH_PREC_F32X2
    from paper_2305_01537_gb300.autograd import chain_loss
    wl = W.chain_8field()
    g = wl.grids[0]
    x = torch.from_numpy(wl.state() * 0.1).cuda()
    w = torch.from_numpy(W.chain_weights(g)).cuda()
    plan = Plan.from_grid(g, precision=SPH_PREC_F32X2 if precision == "f32x2" else SPH_PREC_F64)
    stream = torch.cuda.current_stream()

    def step():
        xd = x.detach().requires_grad_(True)
        chain_loss(xd, plan, w, 8).backward()

    n0 = plan.launch_count
    ms = _timed(step, steps, warmup, stream)
    per_step = (plan.launch_count - n0) / (steps + warmup)
    return {"workload": wl.name, "precision": precision, "value": g.points * 16 * steps / (ms * 1e-3) / 1e9,
            "unit": "Gpoints/s (8 forward + 8 adjoint filter applications per step)", "ms_per_step": ms / steps,
            "gpu_launches_per_step": per_step, "status_ok": plan.sync_status() == 0, "steps": steps}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="f64", choices=list(PRECISIONS),
                    help="arithmetic of the headline line (FP64 by default); the others are timed as variants")
    ap.add_argument("--no-variants", action="store_true", help="time the headline precision only")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the other configurations (256x128x256 state, six-grid batch, differentiable chain)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="state28_128x64x128",
                    choices=["state28_128x64x128", "state28_256x128x256", "batch6_uneven", "chain8_128x64x128",
                             "state28_32x128x256", "hybrid28_128x64x128", "hybrid28_256x128x256",
                             "hybrid28_32x128x256", "constraints_256x64x128"])
    ap.add_argument("--autotune", action="store_true", help="autotune the plan's launch shape before timing")
    ap.add_argument("--inplace", action="store_true",
                    help="filter the state in place (out = in): only the rows a pass transforms are moved")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch6_uneven":
        return run_batch(args)
    if args.workload == "chain8_128x64x128":
        return run_chain(args)
    if args.workload == "constraints_256x64x128":
        return run_constraints(args)

    import torch
    import torch.distributed as dist
    from paper_2305_01537_gb300 import Plan, SPH_PREC_F64, SPH_PREC_F32X2, SPH_PREC_SPLIT_TC, SPH_PREC_SPECTRAL

    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    prec_code = {"f64": SPH_PREC_F64, "f32x2": SPH_PREC_F32X2, "tc": SPH_PREC_SPLIT_TC, "spectral": SPH_PREC_SPECTRAL}

    wl = single_grid_workload(args.workload)
    g = wl.grids[0]
    if W.HYBRID in g.kind:
        variants = [p for p in ("f64", "f32x2") if p != args.precision]  # no hybrid tensor-core form
    else:
        variants = [p for p in PRECISIONS if p != args.precision]
    if args.no_variants or world > 1:
        variants = []
    x_host = torch.from_numpy(wl.state()).pin_memory()
    x = x_host.cuda()
    y = x if args.inplace else torch.empty_like(x)
    plan = Plan.from_grid(g, precision=prec_code[args.precision])
    if args.autotune:
        plan.autotune(x, y)
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            dist.barrier()

    clk = ClockSampler(local).__enter__()
    time.sleep(0.5)  # let nvidia-smi start sampling before the warm-up
    for _ in range(args.warmup):
        plan.apply(x, out=y)
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    wall0 = time.time()
    elapsed_ms, kernel_ms, launched = time_plan(plan, x, y, args.steps, 0, stream)
    barrier()
    wall1 = time.time()
    clk.mark(wall0, wall1)
    assert plan.sync_status() == 0
    y_primary = y.clone() if (world == 1 and not args.no_cpu_baseline and not args.inplace) else None

    # end to end through the host-buffer entry point
    out_host = torch.empty_like(x_host).pin_memory()
    for _ in range(args.warmup):
        plan.apply_host(x_host, out_host)
    torch.cuda.synchronize()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        plan.apply_host(x_host, out_host)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    e2e_ms = e0.elapsed_time(e1)
    copies = host_copy_ceiling(x_host, stream, torch.cuda.Stream()) if rank == 0 else None

    # the other precisions on the same state, for the same line (rank 0 alone, N = 1)
    var_runs = {}
    from paper_2305_01537_gb300 import SphFilterError
    for p in variants:
        try:
            vplan = Plan.from_grid(g, precision=prec_code[p])
        except SphFilterError:  # a form that does not run this shape (the spectral form: one-CTA shells)
            continue
        vy = x.clone() if args.inplace else torch.empty_like(x)
        xin = vy if args.inplace else x
        v_elapsed, v_kernel_ms, v_launched = time_plan(vplan, xin, vy, args.steps, args.warmup, stream)
        assert vplan.sync_status() == 0
        if args.inplace:  # the timed applications filtered in place repeatedly: recompute once for the error
            vy.copy_(x)
            vplan.apply(vy, out=vy)
            torch.cuda.synchronize()
        var_runs[p] = (vplan, vy, v_elapsed, v_kernel_ms, v_launched)
    wall_end = time.time()
    clk.__exit__(None, None, None)

    points = g.points
    (elapsed_ms, e2e_ms), (rate, e2e_rate) = combine_ranks([elapsed_ms, e2e_ms], points, args.steps, device="cuda")
    value = rate / 1e9
    e2e_value = e2e_rate / 1e9
    if rank == 0:
        peaks, src = measured_peaks()
        traffic_rec = {}
        tp = os.path.join(ROOT, "profiles", "traffic.json")
        if os.path.exists(tp):
            with open(tp) as f:
                traffic_rec = json.load(f)

        def traffic_for(p):
            fam = "tc" if p == "tc" else "plain"
            frec = traffic_rec.get("families", {}).get(fam, {})
            if frec.get("sources_sha256_16") == kernel_sources_hash(fam):
                return frec.get(f"{p}:{wl.name}")
            return None

        def label_for(p, pl):
            if p == "tc":
                return "tc_pass_kernel: one persistent launch per application (theta tiles, phi tiles, copies)"
            name = {"f64": "F64", "f32x2": "DF", "spectral": "F64, spectral form"}[p]
            uname = {"f64": "F64", "f32x2": "DF", "spectral": "F64"}[p]
            if pl.launches < 3:
                return f"shell_kernel<{name}>"
            return (f"one application: shell_kernel<{name}> over the shells with a theta pass, units_kernel<{uname}> "
                    "over the active ring pairs of the others" + ("" if args.inplace else ", copy_shells_kernel"))

        avg_kernel_s = statistics.mean(kernel_ms) * 1e-3
        hbm_gbs = 16.0 * points / avg_kernel_s / 1e9
        roof = roofline_for(args.precision, g, avg_kernel_s, points, peaks, src, traffic_for(args.precision),
                            label_for(args.precision, plan))
        if W.HYBRID in g.kind:
            roof["flops_note"] = ("hybrid fields counted as exponential ones: a lower bound (the rings and "
                                  "circles where the detector fires are transformed too)")
        ceiling = points / (copies["both_ways_ms"] * 1e-3) / 1e9
        line = {
            "metric": "filtered Gpoints/s (theta+phi double FFT filter, FP64 I/O)",
            "value": value, "unit": "Gpoints/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": DTYPE_NAME[args.precision],
            "data": "synthetic",
            "config": {"workload": wl.name, "Nr": g.Nr, "Ntheta": g.Ntheta, "Nphi": g.Nphi, "nvars": g.nvars,
                       "precision": args.precision,
                       "l2": f"inputs ({8 * points / 1e6:.0f} MB) larger than L2; no flush",
                       "inplace": bool(args.inplace),
                       "parallelism": f"independent shards x{world}"},
            "hbm": {"achieved_gbs": hbm_gbs, "peak_gbs": peaks["hbm_gbs"], "frac": hbm_gbs / peaks["hbm_gbs"],
                    "peak_source": src, "bytes_per_point": 16},
            "roofline": roof,
            "e2e": {"value": e2e_value, "unit": "Gpoints/s", "h2d_bytes_per_step": 8 * points,
                    "d2h_bytes_per_step": 8 * points, "host_copies": copies,
                    "copy_ceiling_gpoints": ceiling, "frac_of_copy_ceiling": e2e_value / ceiling},
            "gpu_launches": launched,
            "clocks": clk.summary(),
        }
        if world == 1 and not args.no_cpu_baseline:
            cpu, idx, ref = cpu_baseline(g, x_host.numpy(), stride0=16 if g.Nr <= 128 else 64)
            line["cpu_baseline"] = cpu
            if y_primary is not None:
                line["max_err_vs_oracle"] = sample_error(y_primary, idx, ref)
        else:
            idx = ref = None
        if var_runs:
            line["variants"] = {}
            for p, (vplan, vy, v_elapsed, v_kernel_ms, v_launched) in var_runs.items():
                v_avg = statistics.mean(v_kernel_ms) * 1e-3
                v_gbs = 16.0 * points / v_avg / 1e9
                line["variants"][p] = {
                    "value": points * args.steps / (v_elapsed * 1e-3) / 1e9, "unit": "Gpoints/s",
                    "ms_per_step": v_elapsed / args.steps, "dtype": DTYPE_NAME[p],
                    "hbm_frac": v_gbs / peaks["hbm_gbs"],
                    "roofline": roofline_for(p, g, v_avg, points, peaks, src, traffic_for(p), label_for(p, vplan)),
                    "max_err_vs_oracle": sample_error(vy, idx, ref) if ref is not None else None,
                    "err_sample": cpu["sample"] if ref is not None else None,
                    "gpu_launches": v_launched,
                    "clocks": clk.summary((wall1, wall_end)),
                }
        if world == 1 and not args.no_extra and args.workload == "state28_128x64x128":
            # the other configurations, in the same run (fewer steps: each application is longer)
            var_runs.clear()
            x = y = y_primary = None
            torch.cuda.empty_cache()
            k = max(3, min(args.steps, 10))
            line["configs"] = {
                "state28_256x128x256": measure_workload("state28_256x128x256", ["tc", "f32x2", "f64"], k,
                                                        args.warmup, 64),
                "batch6_uneven": measure_batch(k, args.warmup),
                "chain8_128x64x128": {p: measure_chain(p, k, args.warmup) for p in ("f64", "f32x2")},
            }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
