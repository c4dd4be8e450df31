"""Benchmark: dispersion curves per second on GB300.

A step is one MASW evaluation of a whole batch -- Algorithm 1 (the
theoretical dispersion curve of every (model, wavelength) item) followed by
Algorithm 2 (least-squares misfit per model). The default workload is the
ragged batch: 8192 models of 3..30 layers over a half-space, 30..400
log-spaced wavelengths from 1 m to twice the model's total thickness
(1,740,640 items), 10 % of the models with a low-velocity layer, test
velocities 50..1200 m/s in steps of 0.25 (4601 points), FP64 decisions.
Inputs are resident in device memory when the timed region starts; L2 is
flushed (256 MB write) between timed steps.

The same line carries:
- the plain one-curve-per-launch GPU path;
- the end-to-end figure through the C ABI with host buffers: the models and
  the observed curve uploaded, the curves and the misfit read back, every
  step;
- the roofline of the dominant kernel, with clocks sampled during the timed
  steps;
- the CPU oracle on a bounded sample (cpu_baseline), with the CPU-rank
  partition study of Section 3.2.

Extras: the uniform batch measured the same way, the autotuner's plan
against the default, differentiation, inversion, uniform stress, higher
modes, the leaky continuation, the first call, the allocation-free entry
point and serving. ``--impl reference`` times the CPU oracle alone (the
reference arm).

Multi-GPU: one process per GPU (torchrun); each rank evaluates its own
seeded batch (weak scaling, no data-path collective).
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2003_02256_gb300 import sharding  # noqa: E402
from paper_2003_02256_gb300 import workloads as W  # noqa: E402

METRIC = "dispersion curves/sec (model x all lambda) and p50/p99 latency vs plain GPU"
UNIT = "curves/s"
WORKLOADS = {
    "ragged": ("ragged_batch: 8192 models, N~U{3..30} layers + half-space, n_lambda~U{30..400} "
               "log-spaced from 1 m to 2x the model's total thickness (1,740,640 items), 10% of "
               "the models with a low-velocity layer; h~U[1,8] m, beta_1~U[100,250] +U[10,120] "
               "per layer, nu~U[0.25,0.4], rho~U[1700,2100]; c grid 50..1200 m/s step 0.25 "
               "(4601 points); FP64 decisions"),
    "uniform": ("uniform_batch: 1024 models x (8 layers + half-space), h~U[1,8] m, "
                "beta_1~U[100,250] +U[10,120] per layer, nu~U[0.25,0.4], rho~U[1700,2100]; 200 "
                "log-spaced lambda 1..150 m; c grid 50..1200 m/s step 0.25 (4601 points); FP64 "
                "decisions"),
}
DEFAULT_MODELS = {"ragged": 8192, "uniform": 1024}


def make_workload(name: str, n_models: int, rank: int = 0):
    """The seeded batch of one rank (weak scaling: rank r draws its own shard)."""
    if name == "uniform":
        return W.uniform_batch(n_models=n_models, seed=W.SEED + 1000 * rank)
    return W.ragged_batch(n_models=n_models, seed=W.SEED + 3 + 1000 * rank)


# Algorithmic FP64 work of one layer-evaluation (element assembly + one
# Schur step) in flops, 2*DFMA + DMUL + DADD: measured by ncu instruction
# counters on the FP64 element (the counting kernel's certificate before its
# element moved to double-float: 186.6 M DFMA, 143.0 M DMUL, 33.3 M DADD over
# 3,686,400 layer-evaluations of the full 1024-model uniform launch; profiles/).
# Every FP64 kernel runs this arithmetic; it is the per-unit figure of the
# rooflines below.
F_LAYER_FLOPS = 149.1
# FP64 flops the counting kernel executes per layer-evaluation now that the
# element runs in double-float on the FP32 pipe and only the Schur step (and
# the exact conversions) on the FP64 pipe: 55.6 M DFMA, 57.6 M DMUL, 39.9 M
# DADD over the same 3,686,400 layer-evaluations (ncu; profiles/).
F_LAYER_FLOPS_EXECUTED64 = 56.6
# FP32 flops per layer-evaluation of the screen kernel (2*FFMA + FMUL + FADD
# per executed (layer, c) pair: 29.6 FFMA, 54.2 FMUL, 16.4 FADD; ncu
# instruction counters of the 64-model case, profiles/).
F_LAYER_FLOPS_FP32 = 129.8
# DRAM bytes (read + write) of one screen launch per model (ncu, 64-model case:
# 239.6 KB read, 0 written), scaled by the models of a launch.
SCREEN_DRAM_BYTES_PER_MODEL = 239.6e3 / 64
# FP32 pipe: FFMA issue rate per SM per clock.
FP32_FFMA_PER_CLK_SM = 128.0
# FP64 pipe of GB300: DFMA issue rate per SM per clock (ncu peak_sustained) and
# the maximum SM clock.
FP64_DFMA_PER_CLK_SM = 2.0
SM_MAX_MHZ = 2070.0
# DRAM bytes (read + write) of one count_certify launch, from ncu captures
# (dram__bytes_read.sum + dram__bytes_write.sum) of the full workload, as
# (bytes, models of that launch); the records, wavenumbers, item tables and
# the search's indices are read once. Scaled by the models of a launch; None
# where no capture of the current kernel exists.
# uniform: 5.27 MB for the 1024-model launch of count_certify_kernel<128,
# true> (most of its outputs stay in L2); ragged: 49.51 MB for the
# 8192-model launch of count_certify_kernel<256, true> (47.71 MB read,
# 1.80 MB written by the end of the launch).
CERTIFY_DRAM_BYTES = {"uniform": (5.355264e6, 1024), "ragged": (49.506048e6, 8192)}
# Warp instructions a kernel issues per layer-evaluation (ncu
# smsp__inst_executed.sum of one full-workload launch / its layer-evaluations
# counted as in counting_evals), by workload: the certificate kernel per
# certificate layer-evaluation, the search kernels (both passes) per FP32
# one. A kernel's ceiling is the SM's issue rate, ISSUE_PER_CLK_SM warp
# instructions per clock, over this count.
CERTIFY_WARP_INSTR_PER_LAYER_EVAL = {"uniform": 51.25, "ragged": 51.95}
# the split search's anchor stride (SEARCH_STRIDE in csrc/masw_internal.h)
SEARCH_STRIDE = 6
SEARCH_WARP_INSTR_PER_LAYER_EVAL = {"uniform": 8.61, "ragged": 8.21}
ISSUE_PER_CLK_SM = 4
# Warp instructions per layer-evaluation of the leaky continuation's scan
# kernel, element and Schur step in double-float (ncu smsp__inst_executed.sum
# of the 256-model leaky batch's scan launch, 2,242.6 M, over its 50.68 M
# layer-evaluations counted as in extra_leaky); its FP64 pipe is 31 % busy.
LEAKY_WARP_INSTR_PER_LAYER_EVAL = 2242.64e6 / 50.68e6
# DRAM bytes (read + write) of one scan launch per model, from the ncu capture
# of the 64-model case (281.6 KB read, 0 written), scaled by the models of a
# launch; traffic grows with the number of items.
SCAN_DRAM_BYTES_PER_MODEL = 281.6e3 / 64


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), \
        int(os.environ.get("LOCAL_RANK", 0))


class ClockSampler:
    """SM clocks and clock-event (throttle) reasons sampled during the timed
    region: through NVML (read-only queries, every 2 ms, on a host thread)
    when libnvidia-ml loads, else through nvidia-smi every 200 ms."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    # clock-event reason bits of NVML's public header
    NVML_REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
                    0x40: "hw_thermal_slowdown"}
    NVML_CLOCK_SM = 1

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.lines = []
        self.nvml = None
        self.samples = []  # (sm MHz, max MHz, reason bits)
        self.stop = threading.Event()

    def _nvml_open(self):
        try:
            lib = ctypes.CDLL("libnvidia-ml.so.1")
            if lib.nvmlInit_v2() != 0:
                return None
            h = ctypes.c_void_p()
            if lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(self.gpu), ctypes.byref(h)) != 0:
                return None
            reasons = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                getattr(lib, "nvmlDeviceGetCurrentClocksThrottleReasons", None)
            if reasons is None:
                return None
            return lib, h, reasons
        except (OSError, AttributeError):
            return None

    def _nvml_loop(self):
        lib, h, reasons = self.nvml
        clk, mx, bits = ctypes.c_uint(), ctypes.c_uint(), ctypes.c_ulonglong()
        while not self.stop.is_set():
            if (lib.nvmlDeviceGetClockInfo(h, self.NVML_CLOCK_SM, ctypes.byref(clk)) == 0 and
                    lib.nvmlDeviceGetMaxClockInfo(h, self.NVML_CLOCK_SM, ctypes.byref(mx)) == 0 and
                    reasons(h, ctypes.byref(bits)) == 0):
                self.samples.append((clk.value, mx.value, bits.value))
            time.sleep(0.002)

    def __enter__(self):
        self.nvml = self._nvml_open()
        if self.nvml is not None:
            self.t = threading.Thread(target=self._nvml_loop, daemon=True)
            self.t.start()
            return self
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.nvml is not None:
            self.stop.set()
            self.t.join(timeout=5)
            self.nvml[0].nvmlShutdown()
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.samples:
            sm = [x[0] for x in self.samples]
            reasons = {n for b, n in self.NVML_REASONS.items()
                       if any(x[2] & b for x in self.samples)}
            return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(x[1] for x in self.samples)),
                    "reasons": sorted(reasons), "samples": len(sm), "source": "nvml, every 2 ms"}
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)),
                "reasons": sorted(reasons), "samples": len(sm), "source": "nvidia-smi, every 200 ms"}


def cpu_oracle_rate(models, grid, sample, threads: int = 0, banded: bool = False):
    """Time the CPU oracle (dense LU), or with banded=True the CPU banded
    baseline (the paper's serial banded elimination restated), on the models
    with indices ``sample`` of the workload, on `threads` host threads (0: all
    cores). Returns (curves/s, threads, sample description)."""
    import oracle
    oracle.build()
    cores = threads or os.cpu_count() or 1
    sample = np.asarray(sample)
    sub = models.subset(sample)
    run = oracle.dispersion_banded if banded else oracle.dispersion
    t0 = time.perf_counter()
    run(sub.as_dict(), grid.c0, grid.dc, grid.n_c, n_threads=cores)
    dt = time.perf_counter() - t0
    step = int(sample[1] - sample[0]) if sample.size > 1 else 1
    return sample.size / dt, cores, (f"{sample.size} of the {models.n_models} models (every "
                                     f"{step}th from {int(sample[0])}), all their wavelengths "
                                     f"({sub.n_items} items), {dt:.1f} s on {cores} threads")


def _partition_rank(rank, world, reps, barrier, queue):
    """One CPU rank of the partition study: Algorithm 1 with the oracle on its
    share of the 40 wavelengths of the variable curve, for each partition,
    timed between two barriers (the same start for every rank)."""
    import oracle
    m, g = W.single_curve()
    h, a, b, r, _ = m.model(0)
    lam = sharding.variable_curve_wavelengths(40)
    out = {}
    for mode in ("contiguous", "modular"):
        mine = sharding.shard(lam.size, rank, world, mode)
        times = []
        for _ in range(3):
            barrier.wait()
            t0 = time.perf_counter()
            for _ in range(reps):
                idx = [oracle.scan(h, a, b, r, lam[i], g.c0, g.dc, g.n_c)[2] for i in mine]
            times.append(time.perf_counter() - t0)
        out[mode] = (times, mine.tolist(), idx)
    queue.put((rank, out))


def cpu_partition_study(ranks=(1, 2, 3, 4, 8, 16), reps: int = 20):
    """Section 3.2 on CPU ranks: the 40-wavelength decreasing curve split over
    P spawned processes (contiguous blocks or the paper's modular partition),
    each running the oracle's Algorithm 1 on its share ``reps`` times; the
    wall time of a run is that of the slowest rank (median of 3 runs), and
    the speedup is the one-rank time over it. Beside it, the cost model
    (total work over the busiest rank's, work = determinants evaluated)."""
    import multiprocessing as mp
    import oracle
    oracle.build()
    ctx = mp.get_context("spawn")
    cores = os.cpu_count() or 1
    m, g = W.single_curve()
    h, a, b, r, _ = m.model(0)
    lam = sharding.variable_curve_wavelengths(40)
    serial_idx = [oracle.scan(h, a, b, r, l, g.c0, g.dc, g.n_c)[2] for l in lam]
    work = np.asarray(serial_idx, dtype=np.float64) + 1.0
    res = {}
    for P in ranks:
        if P > cores:
            continue
        barrier, queue = ctx.Barrier(P), ctx.Queue()
        procs = [ctx.Process(target=_partition_rank, args=(q, P, reps, barrier, queue))
                 for q in range(P)]
        for p in procs:
            p.start()
        got = [queue.get(timeout=600) for _ in range(P)]
        for p in procs:
            p.join(timeout=60)
        row = {}
        for mode in ("contiguous", "modular"):
            idx = np.full(lam.size, -1)
            for _, out in got:
                idx[out[mode][1]] = out[mode][2]
            assert np.array_equal(idx, serial_idx), "gathered indices differ from one rank's"
            wall = [max(out[mode][0][k] for _, out in got) for k in range(3)]
            row[mode] = {"wall_s": float(np.median(wall)),
                         "cost_model_speedup": sharding.partition_speedup(work, P, mode)}
        res[P] = row
    t1 = np.median([res[1][mode]["wall_s"] for mode in ("contiguous", "modular")])
    for P, row in res.items():
        for mode in row:
            row[mode]["speedup"] = float(t1 / row[mode]["wall_s"])
    return {"workload": "single-curve model (4 layers + half-space, c grid 50..500 step 0.5), "
                        f"40 log-spaced decreasing wavelengths 60..1 m, Algorithm 1 x {reps} per "
                        "run on each rank's share; ranks = spawned processes, one per core",
            "cores": cores,
            "ranks": {str(P): row for P, row in res.items()},
            "paper_section_3_2": {"3": {"modular": 2.8, "contiguous": 1.9},
                                  "8": {"modular": 7.0, "contiguous": 4.2}}}


def run_reference(args):
    """The reference arm: the CPU oracle (Algorithm 1 by dense LU, all host
    cores) on the same workload, metric and unit; each step a bounded sample
    of the workload's models (strided through the batch)."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    n_models = args.models or DEFAULT_MODELS[args.workload]
    models, grid = make_workload(args.workload, n_models, 0)
    per_step = 16
    stride = max(1, n_models // (per_step * max(1, args.steps)))
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    for w in range(args.warmup):
        sub = models.subset(range(w, min(n_models, w + 4)))
        oracle.dispersion(sub.as_dict(), grid.c0, grid.dc, grid.n_c, n_threads=cores)
    times = []
    for s in range(args.steps):
        ms = [(s * per_step + q) * stride % n_models for q in range(per_step)]
        sub = models.subset(ms)
        t0 = time.perf_counter()
        oracle.dispersion(sub.as_dict(), grid.c0, grid.dc, grid.n_c, n_threads=cores)
        times.append(time.perf_counter() - t0)
    value = per_step * args.steps / sum(times)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * float(np.mean(times)), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload], "sample_models_per_step": per_step},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{per_step} models per step (every {stride}th model), "
                                       "all their wavelengths"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def algorithmic_layer_evals(models, idx, st, nlim):
    """Sum over items of (evaluated grid points) x (N + 1): idx + 1 points
    when a root is found, the whole scannable range otherwise."""
    nl = np.repeat(models.n_layers.astype(np.int64) + 1, models.n_lambda)
    pts = np.where(st == 0, idx.astype(np.int64) + 1, np.repeat(nlim, models.n_lambda))
    return int(np.sum(pts * nl))


def executed_layer_evals(models, idx, st, nlim, cpl):
    """Layer evaluations the scan kernel actually executes: whole 32*cpl
    chunks up to the one holding the root, lanes past the scan limit idle."""
    nl = np.repeat(models.n_layers.astype(np.int64) + 1, models.n_lambda)
    lim = np.repeat(nlim, models.n_lambda).astype(np.int64)
    chunk = 32 * cpl
    last = np.where(st == 0, idx.astype(np.int64), lim - 1)
    pts = np.minimum((last // chunk + 1) * chunk, lim)
    return int(np.sum(pts * nl))


def _bisect_evals(lo, hi, r, active):
    """Evaluations of the bisection of (lo, hi] (count 0 at lo, nonzero at
    hi) down to the first nonzero point r, item by item (numpy arrays)."""
    ev = np.zeros_like(lo)
    lo, hi = lo.copy(), hi.copy()
    act = active & (hi - lo > 1)
    while act.any():
        mid = lo + ((hi - lo) >> 1)
        ev += act
        up = mid >= r
        hi = np.where(act & up, mid, hi)
        lo = np.where(act & ~up, mid, lo)
        act &= hi - lo > 1
    return ev


def split_search_evals(models, npf, root, stride=None):
    """FP32 evaluations per item of the split search (count_search_kernel),
    simulated step by step on a count that turns nonzero at the item's first
    change (root, when it lies inside the pole-free range): every stride-th
    item of a model and its last bisect the range, evaluating its top only
    when the bisection ends there (count_search_single); the others start from the guess of search_guess
    (the line through those neighbours' indices, rounded down from a quarter
    point below it), step away from it by 1, 2, 4, ... points until the
    change is bracketed, and bisect the bracket (count_search_guess)."""
    stride = stride or SEARCH_STRIDE
    n_items = models.n_items
    woff = np.concatenate([[0], np.cumsum(models.n_lambda)])
    item_model = np.repeat(np.arange(models.n_models), models.n_lambda)
    j = np.arange(n_items)
    first, last = woff[item_model], woff[item_model + 1] - 1
    npf = np.asarray(npf, dtype=np.int64)
    r = np.where(root < npf, root, -1).astype(np.int64)
    has = npf >= 1
    # single: bisection of (-1, npf - 1], the top evaluated when it ends there
    r_none = np.where(r >= 0, r, np.iinfo(np.int64).max)
    full = (_bisect_evals(np.full(n_items, -1, np.int64), npf - 1, r_none, has)
            + (has & ((r < 0) | (r == npf - 1))))
    ja = first + ((j - first) // stride) * stride
    jb = np.minimum(ja + stride, last)
    anchor = ((j - first) % stride == 0) | (j == last)
    na, nb = r[ja], r[jb]
    guess = has & ~anchor & (na >= 1) & (nb >= 1)
    lin = na + (nb - na) * (j - ja) / np.maximum(jb - ja, 1)
    g = np.clip(np.floor(lin - 0.25).astype(np.int64), 0, np.maximum(npf - 1, 0))
    ev = guess.astype(np.int64)
    down = guess & (r >= 0) & (r <= g)
    up = guess & ~down
    lo = np.where(down, -1, g)
    hi = np.where(down, g, -1)
    step = 1
    act_d = down & (hi > 0)
    act_u = up & (lo < npf - 1)
    while act_d.any() or act_u.any():
        pd = np.maximum(hi - step, 0)
        pu = np.minimum(lo + step, npf - 1)
        ev += act_d | act_u
        zero_d = pd < r  # count 0 at pd: the bracket's lower end
        lo = np.where(act_d & zero_d, pd, lo)
        hi = np.where(act_d & ~zero_d, pd, hi)
        act_d &= ~zero_d & (hi > 0)
        hit_u = (r >= 0) & (pu >= r)
        hi = np.where(act_u & hit_u, pu, hi)
        lo = np.where(act_u & ~hit_u, pu, lo)
        act_u &= ~hit_u & (lo < npf - 1)
        step *= 2
    ev += _bisect_evals(lo, hi, r, guess & (hi >= 0))
    return np.where(has, np.where(guess, ev, full), 0)


def counting_evals(models, grid, idx, st, nlim, n32, split=True):
    """Per-item evaluations of the counting-search scan (plan precision 2).
    FP32 layer evaluations of the search, npf = grid points below the
    pole-free bound min_i beta_i sqrt(1 + (pi/(k h_i))^2): split (its own
    kernels, one thread per item) as split_search_evals; fused (a lane pair)
    1 + ceil(log3 npf) steps of two inertia counts. FP64 layer evaluations of
    the certificate: 2 per counted item. Fallback items: the linear FP32
    scan from its start up to the change, and the three-point FP64 check."""
    counted = (n32 >= 0) & ((n32 & (1 << 30)) != 0)
    item_model = np.repeat(np.arange(models.n_models), models.n_lambda)
    nl = (models.n_layers.astype(np.int64) + 1)[item_model]
    k = 2.0 * np.pi / models.lam
    cb = np.full(models.n_items, np.inf)
    woff = np.concatenate([[0], np.cumsum(models.n_lambda)])
    for m in range(models.n_models):
        h, _, b, _, _ = models.model(m)
        sl = slice(int(woff[m]), int(woff[m + 1]))
        kk = k[sl][:, None]
        cb[sl] = np.min(b[None, :-1] * np.sqrt(1.0 + (np.pi / (kk * h[None, :])) ** 2), axis=1)
    lim = nlim[item_model].astype(np.int64)
    npf = np.clip(np.ceil((cb * (1.0 - 1e-4) - grid.c0) / grid.dc), 0, lim).astype(np.int64)
    root = np.where(st == 0, idx.astype(np.int64), lim - 1)
    if split:
        search = split_search_evals(models, npf, root)
    else:
        steps = np.where(npf >= 2, 1 + np.ceil(np.log(np.maximum(npf, 2)) / np.log(3.0)), 1)
        search = np.where(npf >= 1, 2 * steps, 0)
    start = np.where(root >= npf, npf, 0)
    linear = np.where(counted, 0, np.maximum(root - start + 1, 0))
    live = lim >= 2
    e32 = int(np.sum(np.where(live, search + linear, 0) * nl))
    e64_counted = int(np.sum(np.where(live & counted, 2, 0) * nl))
    e64_fallback = int(np.sum(np.where(live & ~counted, 3, 0) * nl))
    return e32, e64_counted, e64_fallback, float(np.mean(counted))


def counting_roofline(models, grid, idx, st, nlim, n32, phases, peak64, micro, sms, workload):
    """Roofline of the dominant kernel of a counting-search scan, the FP64
    certificate (count_certify_kernel; with the fused plan, the search runs
    inside it): its FP64 work (2 layer-evaluation chains per counted item)
    against the FP64 pipe, from algorithmic layer evaluations / device time.
    The FP32 search's work is reported against the FP32 pipe, over its own
    kernel's time when it has one. Also the linear scan's count (Algorithm
    1's (idx + 1)(N + 1) layer-evaluations per item) and how much of it the
    counting search leaves out."""
    split = phases[3] is not None
    e32, e64, e64_fb, frac_counted = counting_evals(models, grid, idx, st, nlim, n32, split)
    linear = algorithmic_layer_evals(models, idx, st, nlim)
    peak32 = FP32_FFMA_PER_CLK_SM * 2.0 * sms * SM_MAX_MHZ * 1e6
    t0 = (phases[4] if split else phases[0]) * 1e-3
    t32 = (phases[3] if split else phases[0]) * 1e-3
    achieved = e64 * F_LAYER_FLOPS / t0
    cap = CERTIFY_DRAM_BYTES.get(workload)
    wi = CERTIFY_WARP_INSTR_PER_LAYER_EVAL.get(workload) if split else None
    # the roof: the FP64 pipe for the plain FP64 element and step, the SM's
    # instruction issue for the double-float form (its instruction mix
    # measured by ncu); both in the algorithmic flops of a layer-evaluation
    peak_issue = (ISSUE_PER_CLK_SM * sms * SM_MAX_MHZ * 1e6 / wi * F_LAYER_FLOPS) if wi else None
    roof = peak_issue if peak_issue else peak64
    kernel = ("count_certify_kernel (FP64 certificate: double-float element on the FP32 pipe, "
              "Schur step on the FP64 pipe; the FP32 search in count_search_kernel before it)"
              if split else
              "count_certify_kernel (FP64 certificate: double-float element on the FP32 pipe, "
              "Schur step on the FP64 pipe; FP32 search alongside)")
    return {"bound": "alu", "unit": "TFLOP/s",
            "achieved": achieved / 1e12, "peak": roof / 1e12, "frac": achieved / roof,
            "traffic": None if cap is None else cap[0] * models.n_models / cap[1],
            "kernel": kernel,
            "work": "the certificate's layer-evaluations x the FP64 element + Schur step's "
                    "149.1 flops each",
            "peak_source": ("derived: 4 warp instructions issued/clk/SM x SMs x 2070 MHz / "
                            f"{wi} warp instructions per layer-evaluation (ncu) x 149.1 flops"
                            if peak_issue else
                            "derived: 2 DFMA/clk/SM x 2 flop x SMs x 2070 MHz"),
            "warp_instructions_per_layer_eval": wi,
            "fp64_peak": peak64 / 1e12, "frac_of_fp64_peak": achieved / peak64,
            "frac_of_fp64_microbenchmark": achieved / micro,
            "layer_evals_per_launch": e64, "flops_per_layer_eval": F_LAYER_FLOPS,
            "layer_evals_per_s": e64 / t0,
            "fp64_flops_executed_per_layer_eval": F_LAYER_FLOPS_EXECUTED64,
            "fp64_pipe_frac_executed": e64 * F_LAYER_FLOPS_EXECUTED64 / t0 / peak64,
            "kernel_ms": t0 * 1e3,
            "search_layer_evals_fp32": e32,
            "search_fp32_frac_of_fp32_peak": e32 * F_LAYER_FLOPS_FP32 / t32 / peak32,
            "search_frac_of_issue_ceiling": (
                e32 / t32 / (ISSUE_PER_CLK_SM * sms * SM_MAX_MHZ * 1e6 /
                             SEARCH_WARP_INSTR_PER_LAYER_EVAL[workload])
                if split and workload in SEARCH_WARP_INSTR_PER_LAYER_EVAL else None),
            "fallback_check_layer_evals_fp64": e64_fb,
            "linear_scan_layer_evals": linear,
            "linear_scan_over_counting_evals": linear / max(1, e32 + e64 + e64_fb),
            "phases_ms": {"count_search_and_certify": phases[0],
                          "count_search": phases[3], "count_certify": phases[4],
                          "fallback_check_search": phases[1], "resolve64": phases[2],
                          "fallback_chain_beside_certificate": phases[5]},
            "counted_fraction": frac_counted,
            "fp64_peak_microbenchmark": micro / 1e12}


def device_steps(torch, step, steps, flush, stream, after=None):
    """CUDA-event times (ms) of ``steps`` calls of ``step`` on ``stream``, L2
    flushed before each; ``after`` is called after each step has finished."""
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    for k in range(steps):
        flush.zero_()
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
        torch.cuda.synchronize()
        if after:
            after()
    return [a.elapsed_time(b) for a, b in ev]


def kernel_phases(torch, masw, batch, step, steps, flush, stream):
    """Per-kernel device times of the scan (ms, mean over ``steps`` timed
    steps): the same kernels launched without the graph, so that CUDA events
    on the batch stream sit between them (masw_last_scan_phases, and
    masw_last_count_phases for the split counting kernels). Returns the three
    scan phases, then the search and certificate kernels and the fallback
    chain on the second stream (None when fused; 0 without the second
    stream)."""
    plan = batch.plan()
    batch.set_plan(use_graph=0)
    split = plan.precision == 2 and plan.count_split >= 1
    ph = []
    device_steps(torch, step, steps, flush, stream,
                 after=lambda: ph.append(masw.last_scan_phases(batch.handle) +
                                         (masw.last_count_phases(batch.handle) if split
                                          else [None, None, None])))
    batch.set_plan(use_graph=plan.use_graph)
    return [None if ph[0][i] is None else float(np.mean([p[i] for p in ph])) for i in range(6)]


def e2e_rate(torch, masw, models, grid, ce_host, plan, steps, warmup, n_pipe):
    """End to end through the C ABI with host buffers, every step: the models
    (h, alpha, beta, rho) and the observed curve C_e uploaded from pinned host
    memory (masw_model_batch_update, masw_misfit_curves), Algorithms 1 and 2,
    and the curves (C_t, index, status) and the misfit read back into pinned
    host memory. With n_pipe > 1 the steps alternate between n_pipe batches,
    each on its own stream and host thread, so one step's copies overlap
    another's kernels. Returns (curves/s, H2D bytes, D2H bytes per step)."""
    import threading
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    hh, ha, hb, hr, hce = (pin(x) for x in (models.h, models.alpha, models.beta, models.rho,
                                            ce_host))
    streams = [torch.cuda.Stream() for _ in range(n_pipe)]
    batches = [masw.Batch(models, grid, stream=st.cuda_stream) for st in streams]
    outs = []
    for b in batches:
        masw.set_plan(b.handle, plan)
        outs.append((torch.empty(models.n_models, dtype=torch.float64).pin_memory(),
                     torch.empty(models.n_items, dtype=torch.float64).pin_memory(),
                     torch.empty(models.n_items, dtype=torch.int32).pin_memory(),
                     torch.empty(models.n_items, dtype=torch.int32).pin_memory()))

    def one(q):
        masw.model_batch_update(batches[q].handle, hh, ha, hb, hr)
        masw.misfit_curves(batches[q].handle, hce, masw.MISFIT_LSQ, 2.0, *outs[q])

    for _ in range(warmup):
        for q in range(n_pipe):
            one(q)
    torch.cuda.synchronize()
    go = threading.Barrier(n_pipe + 1)
    errors = []

    def worker(q):
        go.wait()
        try:
            for _ in range(q, steps, n_pipe):
                one(q)
        except Exception as e:  # surfaced after the join
            errors.append(e)

    threads = [threading.Thread(target=worker, args=(q,)) for q in range(n_pipe)]
    for t in threads:
        t.start()
    go.wait()
    t0 = time.perf_counter()
    for t in threads:
        t.join()
    elapsed = time.perf_counter() - t0
    if errors:
        raise errors[0]
    for b in batches:
        b.close()
    elapsed = sharding.max_over_ranks(elapsed, device="cuda")
    h2d = sum(x.numel() * x.element_size() for x in (hh, ha, hb, hr, hce))
    d2h = sum(x.numel() * x.element_size() for x in outs[0])
    return models.n_models * steps / elapsed, h2d, d2h


def measure(args, torch, masw, workload, n_models, rank, world, with_plain=True):
    """The whole measurement of one workload: device-timed steps (value),
    clocks, per-kernel times and the roofline of the dominant kernel, the
    plain one-curve-per-launch path and the end-to-end figures."""
    stream = torch.cuda.current_stream()
    models, grid = make_workload(workload, n_models, rank)
    ce_host = W.noisy_observation(np.full(models.n_items, 250.0), sigma=30.0, seed=rank)
    batch = masw.Batch(models, grid)
    if args.precision is not None:
        batch.set_plan(precision=args.precision)
    if args.cpl is not None:
        batch.set_plan(cpl=args.cpl)
    plan = batch.autotune(reps=3) if args.autotune else batch.plan()

    # results of one pass (parity-checked in tests; used for the algorithmic count)
    ct, idx, st = batch.dispersion()
    bhs = np.array([models.model(q)[2][-1] for q in range(models.n_models)])
    nlim = np.searchsorted(grid.c0 + grid.dc * np.arange(grid.n_c), bhs, side="left")
    n32 = None
    if plan.precision >= 1:
        n32 = np.empty(models.n_items, dtype=np.int32)
        masw.last_scan_screen(batch.handle, n32)
    unresolved = batch.last_scan_unresolved()
    fallback = batch.last_scan_fallback()

    ce = torch.from_numpy(ce_host).cuda()
    phi = torch.empty(models.n_models, dtype=torch.float64, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def step():
        masw.misfit(batch.handle, ce, masw.MISFIT_LSQ, 2.0, phi)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    scan_ms = []
    with ClockSampler(torch.cuda.current_device()) as clk:
        step_ms = device_steps(torch, step, args.steps, flush, stream,
                               after=lambda: scan_ms.append(batch.last_scan_ms()))
    total_ms = sharding.max_over_ranks(float(np.sum(step_ms)), device="cuda")
    value = world * models.n_models * args.steps / (total_ms * 1e-3)

    # per-kernel times over the same number of timed steps, graph-free
    phases = kernel_phases(torch, masw, batch, step, args.steps, flush, stream) \
        if plan.precision >= 1 else None

    with ClockSampler(torch.cuda.current_device()) as clk_micro:
        micro = float(np.median([masw.fp64_peak() for _ in range(3)]))
    sms = masw.sm_count()
    peak = FP64_DFMA_PER_CLK_SM * 2.0 * sms * SM_MAX_MHZ * 1e6
    units = algorithmic_layer_evals(models, idx, st, nlim)
    if plan.precision == 2:
        roofline = counting_roofline(models, grid, idx, st, nlim, n32, phases, peak, micro, sms,
                                     workload)
        roofline.update({"scan_ms": float(np.mean(scan_ms)), "unresolved_items": unresolved,
                         "fallback_items": fallback,
                         "fp64_peak_microbenchmark_clocks": clk_micro.summary()})
    elif plan.precision == 0:
        scan_avg = float(np.mean(scan_ms)) * 1e-3
        achieved = units * F_LAYER_FLOPS / scan_avg
        roofline = {"bound": "alu", "achieved": achieved / 1e12, "peak": peak / 1e12,
                    "unit": "TFLOP/s", "frac": achieved / peak,
                    "traffic": SCAN_DRAM_BYTES_PER_MODEL * models.n_models,
                    "kernel": "scan_kernel (FP64 pipe)",
                    "peak_source": "derived: 2 DFMA/clk/SM x 2 flop x SMs x 2070 MHz",
                    "peak_microbenchmark": micro / 1e12,
                    "layer_evals_per_launch": units, "flops_per_layer_eval": F_LAYER_FLOPS,
                    "executed_layer_evals_per_launch":
                        executed_layer_evals(models, idx, st, nlim, plan.cpl),
                    "scan_ms": scan_avg * 1e3}
    else:
        peak32 = FP32_FFMA_PER_CLK_SM * 2.0 * sms * SM_MAX_MHZ * 1e6
        t_screen = phases[0] * 1e-3
        achieved = units * F_LAYER_FLOPS_FP32 / t_screen
        roofline = {"bound": "alu", "achieved": achieved / 1e12, "peak": peak32 / 1e12,
                    "unit": "TFLOP/s", "frac": achieved / peak32,
                    "traffic": SCREEN_DRAM_BYTES_PER_MODEL * models.n_models,
                    "kernel": "screen32_kernel (FP32 pipe)",
                    "peak_source": "derived: 128 FFMA/clk/SM x 2 flop x SMs x 2070 MHz",
                    "layer_evals_per_launch": units,
                    "flops_per_layer_eval": F_LAYER_FLOPS_FP32,
                    "scan_ms": float(np.mean(scan_ms)),
                    "phases_ms": {"screen32": phases[0], "check_search": phases[1],
                                  "resolve64": phases[2]},
                    "fp64_peak_derived": peak / 1e12, "fp64_peak_microbenchmark": micro / 1e12,
                    "unresolved_items": unresolved}

    # plain one-curve-per-launch path (one launch + sync per model)
    plain = None
    if with_plain and not args.no_plain:
        plain_ms = []
        for _ in range(2):
            t0 = time.perf_counter()
            batch.dispersion(plain=True)
            plain_ms.append(1e3 * (time.perf_counter() - t0))
        pv = models.n_models / (min(plain_ms) * 1e-3)
        plain = {"value": pv, "unit": UNIT, "ms_per_step": min(plain_ms),
                 "speedup_of_batched": value / world / pv}

    # end to end through the C ABI with host buffers: pipelined (the line's
    # figure) and one batch on one thread (for the gap)
    e2e_steps = max(args.steps, 2)
    ev_p, h2d, d2h = e2e_rate(torch, masw, models, grid, ce_host, plan, e2e_steps, args.warmup, 2)
    ev_1, _, _ = e2e_rate(torch, masw, models, grid, ce_host, plan, e2e_steps, args.warmup, 1)
    e2e = {"value": world * ev_p, "unit": UNIT, "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": d2h,
           "how": "every step: models + C_e uploaded from pinned host memory, Algorithms 1+2, "
                  "curves (C_t, index, status) + misfit read back to pinned host memory "
                  "(masw_model_batch_update + masw_misfit_curves); steps alternate between 2 "
                  "batches on 2 streams driven by 2 host threads",
           "one_batch_one_thread": world * ev_1,
           "frac_of_device_value": ev_p * world / value}
    batch.close()
    return {"models": models, "grid": grid, "value": value, "total_ms": total_ms,
            "step_ms_median": float(np.median(step_ms)), "clocks": clk.summary(),
            "roofline": roofline, "plan": plan.as_dict(), "plain": plain, "e2e": e2e,
            "found_fraction": float(np.mean(st == 0)),
            "launches_per_step": {0: 2, 1: 5,
                                  2: (6, 8, 12)[plan.count_split]}[plan.precision]}


def run_extras(args, masw, torch):
    """Secondary workloads on the same line."""
    from paper_2003_02256_gb300 import serving
    out = {}
    only = set(args.extras.split(",")) if args.extras else None

    def want(name):
        return only is None or name in only

    other = "uniform" if args.workload == "ragged" else "ragged"
    if want(other + "_batch"):
        r = measure(args, torch, masw, other, DEFAULT_MODELS[other], 0, 1)
        out[other + "_batch"] = {
            "workload": WORKLOADS[other], "value": r["value"], "unit": UNIT,
            "ms_per_step": r["total_ms"] / args.steps, "clocks": r["clocks"],
            "roofline": r["roofline"], "plain_gpu": r["plain"], "e2e": r["e2e"],
            "plan": r["plan"]}
    if want("autotune"):
        out.update(extra_autotune(args, masw, torch))
    if want("differentiation") or want("inversion"):
        out.update(extra_differentiation_inversion(masw, torch))
    if want("uniform_stress"):
        out.update(extra_uniform_stress(masw))
    if want("higher_modes"):
        out.update(extra_higher_modes(masw, torch))
    if want("leaky"):
        out.update(extra_leaky(masw, torch))
    if want("first_call"):
        out.update(extra_first_call(masw))
    if want("noalloc"):
        out.update(extra_noalloc(masw, torch))
    if want("serving"):
        out.update(extra_serving(args, serving, masw))
    return out


def extra_autotune(args, masw, torch):
    """The autotuner's plan against the default plan on the ragged batch:
    median of 10 scans each (CUDA events on the batch stream)."""
    m3, g3 = W.ragged_batch()
    with masw.Batch(m3, g3) as b:
        default = b.plan()

        def med():
            b.dispersion()
            t = []
            for _ in range(10):
                b.dispersion()
                t.append(b.last_scan_ms())
            return float(np.median(t))

        t_default = med()
        t0 = time.perf_counter()
        tuned = b.autotune(reps=3)
        t_tune = time.perf_counter() - t0
        t_tuned = med()
    return {"autotune": {"workload": "ragged_batch (8192 models), scan only, host outputs",
                         "default_plan": default.as_dict(), "default_scan_ms": t_default,
                         "tuned_plan": tuned.as_dict(), "tuned_scan_ms": t_tuned,
                         "tuning_s": t_tune}}


def extra_differentiation_inversion(masw, torch):
    out = {}
    # differentiation batch
    m4, g4, true = W.differentiation_batch()
    gold = np.loadtxt(os.path.join(ROOT, "tests", "golden", "differentiation_true_roots.txt"))
    ce = np.tile(W.noisy_observation(gold[:, 2], sigma=2.0), m4.n_models)
    with masw.Batch(m4, g4) as b:
        b.misfit_grad(ce)
        torch.cuda.synchronize()
        ts = []
        for _ in range(10):
            t0 = time.perf_counter()
            b.misfit_grad(ce)
            ts.append(time.perf_counter() - t0)
        dt = float(np.median(ts))
    out["differentiation"] = {"workload": "512 models x 12 layers, 150 wavelengths, LSQ misfit "
                                          "+ adjoint gradient (beta, h), host outputs",
                              "gradients_per_s": m4.n_models / dt, "ms_per_batch": 1e3 * dt}
    # inversion loops (one inversion per model of the differentiation batch)
    from paper_2003_02256_gb300 import inversion
    with masw.Batch(m4, g4) as b:
        ce_true = np.tile(gold[:, 2], m4.n_models)
        inversion.gradient_inversion(b, ce_true, iters=2)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, _, hist = inversion.gradient_inversion(b, ce_true, iters=10)
        torch.cuda.synchronize()
        t_grad = time.perf_counter() - t0
        inversion.metropolis(b, ce_true, steps=2, step_frac=0.01)  # warm-up (first torch RNG use)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, _, _, acc = inversion.metropolis(b, ce_true, steps=20, step_frac=0.01)
        torch.cuda.synchronize()
        t_mc = time.perf_counter() - t0
    out["inversion"] = {"workload": "512 models x 12 layers, 150 wavelengths, observed curve = "
                                    "true-model roots (tests/golden)",
                        "descent_model_steps_per_s": m4.n_models * 10 / t_grad,
                        "misfit_ratio_after_10_steps": float(np.median(hist[-1] / hist[0])),
                        "metropolis_chain_steps_per_s": m4.n_models * 20 / t_mc,
                        "metropolis_acceptance": float(np.mean(acc))}
    return out


def extra_uniform_stress(masw):
    out = {}
    # uniform-work stress curves: one wavelength repeated per curve, roots
    # near 72 / 238 / 256 m/s
    stress = {}
    for target in W.STRESS_TARGETS:
        row = {}
        for rep in (50, 100, 200, 500):
            sm, sg = W.uniform_stress(target, rep, n_models=256)
            with masw.Batch(sm, sg) as b:
                sct, _, _ = b.dispersion()
                ms = []
                for _ in range(10):
                    b.dispersion()
                    ms.append(b.last_scan_ms())
            row[str(rep)] = {"curves_per_s": sm.n_models / (float(np.median(ms)) * 1e-3),
                             "scan_ms": float(np.median(ms)), "ct": float(sct[0])}
        stress[f"{target:g}"] = row
    out["uniform_stress"] = {"workload": "256 identical curves per case, one wavelength repeated "
                                         "50..500 times (0.5 m or 2000 m on 2-layer models); "
                                         "c grid 50..1200 step 0.25", "targets_m_s": stress}

    return out


def extra_higher_modes(masw, torch):
    out = {}
    # higher modes: the first 3 sign changes per item (FP64 past the first)
    hm, hg = W.uniform_batch()
    with masw.Batch(hm, hg) as b:
        _, hidx, hst, hdl = b.changes(3)
        hms = []
        for _ in range(3):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            b.changes(3)
            hms.append(time.perf_counter() - t0)
    out["higher_modes"] = {"workload": "uniform_batch (1024 models), first 3 sign changes per item, "
                                       "host outputs", "curves_per_s": hm.n_models / min(hms),
                           "ms": 1e3 * min(hms),
                           "changes_found_fraction": float(np.mean(hst == 0)),
                           "roots_fraction_of_found": float(np.mean(hdl[hst == 0] == 1)),
                           "poles_fraction_of_found": float(np.mean(hdl[hst == 0] == -1))}

    return out


def extra_leaky(masw, torch):
    """Leaky continuation: the whole grid with the sign of Re det K. Besides
    the host-output rate, a roofline of the continuation kernel: the
    layer-evaluations the linear scan needs for the items the batch scan
    leaves without a change (from one point below the scan limit to the
    change, or to the end of the grid), over the kernel's device time (CUDA
    events around the device-output call on the batch stream, less the batch
    scan's own event time; the FP64 confirmation of each change and the
    rescans included), against the issue ceiling of the scan kernel's
    instruction mix (element and Schur step in double-float); both in
    F_LAYER_FLOPS per layer-evaluation."""
    out = {}
    lm, lg = W.leaky_batch()
    n_rec = lm.n_layers.astype(np.int64) + 1
    beta_hs = np.array([lm.model(q)[2][-1] for q in range(lm.n_models)])
    grid = lg.c0 + lg.dc * np.arange(lg.n_c)
    nlim = np.searchsorted(grid, beta_hs, side="left")
    item_model = np.repeat(np.arange(lm.n_models), lm.n_lambda)
    with masw.Batch(lm, lg) as b:
        _, lidx, lst = b.leaky()
        _, _, lst1 = b.dispersion()
        lms, lscan, kms = [], [], []
        for _ in range(5):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            b.leaky()
            lms.append(time.perf_counter() - t0)
            lscan.append(b.last_scan_ms())
        d_ct = torch.empty(lm.n_items, dtype=torch.float64, device="cuda")
        d_idx = torch.empty(lm.n_items, dtype=torch.int32, device="cuda")
        d_st = torch.empty(lm.n_items, dtype=torch.int32, device="cuda")
        for _ in range(5):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            masw.dispersion_leaky(b.handle, d_ct, d_idx, d_st)
            e1.record()
            torch.cuda.synchronize()
            kms.append(e0.elapsed_time(e1) - b.last_scan_ms())
    cont = lst1 != 0
    start = np.maximum(nlim[item_model], 1)
    last = np.where(lst == 0, lidx, lg.n_c - 1)
    evals = float(np.sum(((last - start + 2) * n_rec[item_model])[cont]))
    k_ms = float(np.median(kms))
    achieved = evals * F_LAYER_FLOPS / (k_ms * 1e-3) / 1e12
    sms = masw.sm_count()
    ceiling = ISSUE_PER_CLK_SM * sms * SM_MAX_MHZ * 1e6 / LEAKY_WARP_INSTR_PER_LAYER_EVAL
    peak = ceiling * F_LAYER_FLOPS / 1e12
    peak64 = FP64_DFMA_PER_CLK_SM * 2.0 * sms * SM_MAX_MHZ * 1e6 / 1e12
    out["leaky"] = {"workload": lm.meta["workload"] + ", host outputs",
                    "curves_per_s": lm.n_models / min(lms), "ms": 1e3 * min(lms),
                    "batch_scan_ms": float(np.median(lscan)),
                    "continuation_kernel_ms": k_ms,
                    "found_fraction": float(np.mean(lst == 0)),
                    "continued_fraction": float(np.mean(cont)),
                    "roofline": {"bound": "alu", "unit": "TFLOP/s", "achieved": achieved,
                                 "peak": peak, "frac": achieved / peak,
                                 "kernel": "leaky_scan64_kernel (element and Schur step in "
                                           "double-float on the FP32 pipe, the complex half-space "
                                           "pivot in FP64), then leaky_check_kernel (the FP64 "
                                           "step at each change) and the rescans",
                                 "peak_source": "derived: 4 warp instructions issued/clk/SM x SMs "
                                                "x 2070 MHz / "
                                                f"{LEAKY_WARP_INSTR_PER_LAYER_EVAL:.2f} warp "
                                                "instructions per layer-evaluation (ncu) x 149.1 "
                                                "flops",
                                 "layer_evals": evals, "layer_evals_per_s": evals / (k_ms * 1e-3),
                                 "flops_per_layer_eval": F_LAYER_FLOPS,
                                 "frac_of_fp64_peak": achieved / peak64}}
    return out


def extra_first_call(masw):
    out = {}
    # first use: batch creation (upload, records, graph capture) and the first
    # scan of a fresh batch vs the warm median (CUDA context and library
    # already loaded in this process)
    fm, fg = W.uniform_batch()
    t0 = time.perf_counter()
    fb = masw.Batch(fm, fg)
    t1 = time.perf_counter()
    fb.dispersion()
    t2 = time.perf_counter()
    warm = []
    for _ in range(10):
        t3 = time.perf_counter()
        fb.dispersion()
        warm.append(time.perf_counter() - t3)
    fb.close()
    out["first_call"] = {"workload": "uniform_batch (1024 models), default plan, host outputs",
                         "create_ms": 1e3 * (t1 - t0), "first_dispersion_ms": 1e3 * (t2 - t1),
                         "warm_median_ms": 1e3 * float(np.median(warm))}

    return out


def extra_noalloc(masw, torch):
    """The allocation-free entry point (plain FP64 scan, items in natural
    order) against masw_dispersion (default plan, graph-replayed) on the
    largest uniform batch it accepts: 320 models x 200 wavelengths (64,000
    items), device inputs and outputs; median of 5 calls each, CUDA events on
    the current stream."""
    m, g = W.uniform_batch(n_models=320)
    stream = torch.cuda.current_stream()
    arrs = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in
            (m.n_layers.astype(np.int32), m.h, m.alpha, m.beta, m.rho,
             m.n_lambda.astype(np.int32), m.lam)]
    out = [torch.empty(m.n_items, dtype=t, device="cuda")
           for t in (torch.float64, torch.int32, torch.int32)]

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(5):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return float(np.median(ts))

    t_na = timed(lambda: masw.dispersion_noalloc(*arrs, (g.c0, g.dc, g.n_c), *out))
    idx_na = out[1].cpu().numpy()
    with masw.Batch(m, g) as b:
        t_b = timed(lambda: masw.dispersion(b.handle, *out))
        same = bool(np.array_equal(out[1].cpu().numpy(), idx_na))
    return {"noalloc": {"workload": "uniform_batch, 320 models x 200 wavelengths (64,000 items), "
                                    "device inputs and outputs",
                        "noalloc_ms": t_na, "noalloc_curves_per_s": m.n_models / (t_na * 1e-3),
                        "dispersion_ms": t_b, "dispersion_curves_per_s": m.n_models / (t_b * 1e-3),
                        "identical_indices": same,
                        "noalloc_plan": "counting plan, fused search and certificate"}}


def plain_per_request(masw, reqs, arrival_s, grid, limit_s=10.0):
    """The plain per-request path: each request, when it arrives (or when the
    previous one has finished), gets its own batch (masw_model_batch_create),
    one masw_dispersion_plain call (one launch per curve, synchronised) and
    masw_model_batch_destroy. Returns per-request latencies (s); requests not
    started within ``limit_s`` are left out (the count is returned)."""
    hoff, loff, woff = reqs.layer_offsets()
    lat = []
    t0 = time.perf_counter()
    for i in range(reqs.n_models):
        now = time.perf_counter() - t0
        if now > limit_s:
            break
        if arrival_s[i] > now:
            time.sleep(arrival_s[i] - now)
        one = reqs.subset([i])
        with masw.Batch(one, grid) as b:
            b.dispersion(plain=True)
        lat.append(time.perf_counter() - t0 - arrival_s[i])
    return np.asarray(lat), len(lat)


def extra_serving(args, serving, masw):
    """Serving: a seeded random-walk trace (one model per request, 3..30
    layers, 30..400 wavelengths), Poisson arrivals. The full trace
    (``--serving-requests``, 200k by default) is replayed at 1e4 and 1e5 per
    second; the other rates replay a bounded prefix. Beside the continuous-
    batching server: the same trace through a one-slot server (one request at
    a time, on the device path of the server) and through the plain
    per-request path (batch create + masw_dispersion_plain + destroy), both on
    a prefix; and the admission cap binding (a 64 MB cap on the 1e5/s trace)."""
    out = {}
    sampler = W.RandomWalkSampler()
    t0 = time.perf_counter()
    n_full = args.serving_requests
    reqs_full = W.concat([sampler.next() for _ in range(n_full)])
    gen_s = time.perf_counter() - t0
    grid = W.Grid(50.0, 0.25, 4601)
    n_prefix = min(2000, n_full)
    prefix = reqs_full.subset(range(n_prefix))
    rates = {}
    for rate in (1e3, 3e3, 1e4, 3e4, 1e5, 1e6):
        full = rate in (1e4, 1e5)
        reqs = reqs_full if full else prefix
        arr = W.poisson_arrivals(reqs.n_models, rate=rate)
        with serving.Server(grid, max_slots=2048, chunks_per_tick=8,
                            mem_cap_bytes=16 << 30) as srv:
            lat, _, _, _, st = srv.run_trace(reqs, arr)
        row = {"requests": reqs.n_models, "served": serving.latency_summary(lat, arr, reqs.n_models),
               "ticks": st["ticks"], "refused": st["refused"], "max_in_flight": st["max_in_flight"]}
        arr_p = W.poisson_arrivals(n_prefix, rate=rate)
        with serving.Server(grid, max_slots=1, chunks_per_tick=1 << 20) as one_slot:
            lat_1, _, _, _, _ = one_slot.run_trace(prefix, arr_p)
        row["one_slot_server"] = dict(serving.latency_summary(lat_1, arr_p, n_prefix),
                                      requests=n_prefix)
        lat_p, done = plain_per_request(masw, prefix, arr_p, grid)
        row["plain_per_request"] = dict(serving.latency_summary(lat_p, arr_p[:done], done),
                                        requests=done)
        rates[f"{rate:g}"] = row
    # admission by memory: the 1e5/s trace under a 1 MB cap (the trace holds
    # up to ~1000 requests of a few KB each in flight, far below 16 GB)
    cap = 1 << 20
    arr = W.poisson_arrivals(reqs_full.n_models, rate=1e5)
    with serving.Server(grid, max_slots=2048, chunks_per_tick=8, mem_cap_bytes=cap) as srv:
        lat, _, _, _, st = srv.run_trace(reqs_full, arr)
    capped = {"mem_cap_bytes": cap, "rate_per_s": 1e5, "requests": reqs_full.n_models,
              "served": serving.latency_summary(lat, arr, reqs_full.n_models),
              "ticks": st["ticks"], "refused": st["refused"], "max_in_flight": st["max_in_flight"]}
    # where a tick's time goes: the profiled server on the 1e5/s trace and at
    # 1e6/s (the served ceiling), per-tick means of the device parts (CUDA
    # events between them) and of the host's launch, finish and admission
    ticks_prof = {}
    for rate, reqs in ((1e5, reqs_full), (1e6, prefix)):
        arr = W.poisson_arrivals(reqs.n_models, rate=rate)
        with serving.Server(grid, max_slots=2048, chunks_per_tick=8,
                            mem_cap_bytes=16 << 30) as srv:
            srv.profile(True)
            t0 = time.perf_counter()
            lat, _, _, _, st = srv.run_trace(reqs, arr)
            wall = time.perf_counter() - t0
            prof = srv.profile(False)
        n = max(prof["ticks"], 1.0)
        ticks_prof[f"{rate:g}"] = dict(
            {k: v / n for k, v in prof.items() if k != "ticks"}, ticks=prof["ticks"],
            requests=reqs.n_models, wall_ms_per_tick=1e3 * wall / n,
            served=serving.latency_summary(lat, arr, reqs.n_models))
    out["serving"] = {"workload": f"random-walk model evaluations (layers 3..30, wavelengths "
                                  f"30..400), Poisson arrivals, 16 GB admission cap; "
                                  f"{n_full} requests at 1e4 and 1e5 per s, the first "
                                  f"{n_prefix} at the other rates and on the plain arms "
                                  "(one-slot server; per-request batch + masw_dispersion_plain)",
                      "trace_generation_s": gen_s, "rates_per_s": rates,
                      "admission_cap_binding": capped, "tick_profile_ms_per_tick": ticks_prof}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="ragged", choices=["ragged", "uniform"],
                    help="main workload (the line's config)")
    ap.add_argument("--models", type=int, default=None,
                    help="models per GPU (default: the workload's own; smaller only for "
                         "profiler captures)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--autotune", action="store_true",
                    help="autotune the plan before timing (default: the library's plan)")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--extras", default=None,
                    help="comma-separated subset of the extras (uniform_batch or ragged_batch, "
                         "autotune, differentiation, inversion, uniform_stress, higher_modes, "
                         "leaky, first_call, noalloc, serving); default all")
    ap.add_argument("--serving-requests", type=int, default=200000)
    ap.add_argument("--precision", type=int, default=None, choices=[0, 1, 2],
                    help="scan plan: 0 FP64 scan, 1 FP32 screen + FP64 decision, 2 counting "
                         "search + FP64 certificate (default: library)")
    ap.add_argument("--cpl", type=int, default=None, choices=[1, 2, 4],
                    help="scan plan test velocities per lane (2: paired FP32x2 screen)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    from paper_2003_02256_gb300 import masw

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    n_models = args.models or DEFAULT_MODELS[args.workload]
    r = measure(args, torch, masw, args.workload, n_models, rank, world)
    models, grid = r["models"], r["grid"]

    extras = None
    if rank == 0 and world == 1 and not args.no_extras:
        extras = run_extras(args, masw, torch)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        stride = max(1, models.n_models // 256)
        sample = np.arange(0, models.n_models, stride)[:256]
        v, cores, desc = cpu_oracle_rate(models, grid, sample)
        v1, _, desc1 = cpu_oracle_rate(models, grid, sample[:8], threads=1)
        vb, _, desc_b = cpu_oracle_rate(models, grid, sample, banded=True)
        vb1, _, desc_b1 = cpu_oracle_rate(models, grid, sample[:8], threads=1, banded=True)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc,
               "single_thread": {"value": v1, "unit": UNIT, "sample": desc1},
               "banded": {"value": vb, "unit": UNIT, "cores": cores,
                          "kind": "CPU banded elimination (the paper's serial C, sparse variant, "
                                  "restated; pinned to the oracle)",
                          "sample": desc_b,
                          "single_thread": {"value": vb1, "unit": UNIT, "sample": desc_b1}},
               "partition_study": cpu_partition_study()}

    if rank == 0:
        line = {"metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": r["total_ms"] / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": WORKLOADS[args.workload],
                           "models_per_gpu": models.n_models, "items_per_gpu": models.n_items,
                           "seed": int(models.meta.get("seed", W.SEED)),
                           "l2": "flushed between timed steps (256 MB write)",
                           "step": "Algorithm 1 scan of every item + Algorithm 2 misfit",
                           "step_ms_median": r["step_ms_median"],
                           "plan": r["plan"], "parallelism": f"replicas x{world}"},
                "clocks": r["clocks"],
                "e2e": r["e2e"],
                # per step: the scan's kernels (precision 0: scan; 1: screen, check,
                # mode-count search, re-scan; 2: counting search + certificate,
                # fallback scan, check, mode-count search, re-scan) and the misfit
                "gpu_launches": r["launches_per_step"] * args.steps,
                "roofline": r["roofline"],
                "cpu_baseline": cpu,
                "plain_gpu": r["plain"],
                "found_fraction": r["found_fraction"],
                "extras": extras}
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
