"""Benchmark: dispersion curves per second on GB300.

A step is one MASW evaluation of a whole batch -- Algorithm 1 (theoretical
dispersion curve of every (model, wavelength) item) followed by Algorithm 2
(misfit per model) -- on the uniform workload: 1024 models of 8 layers over a
half-space, 200 log-spaced wavelengths 1..150 m, test velocities 50..1200 m/s
step 0.25 (4601 points), FP64. Inputs are resident in device memory when the
timed region starts; L2 is flushed (256 MB write) between timed steps.

Also reported on the same line: the plain one-curve-per-launch GPU path,
the end-to-end figure through the C ABI with host buffers, the roofline of
the scan kernel against the measured FP64 peak, and the CPU oracle on a
bounded sample (``cpu_baseline``). ``--impl reference`` times the CPU oracle
alone (the reference arm).

Multi-GPU: one process per GPU (torchrun); each rank evaluates its own
1024-model batch (weak scaling, no data-path collective).
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
WORKLOAD = ("uniform_batch: 1024 models x (8 layers + half-space), h~U[1,8] m, beta_1~U[100,250] "
            "+U[10,120] per layer, nu~U[0.25,0.4], rho~U[1700,2100]; 200 log-spaced lambda "
            "1..150 m; c grid 50..1200 m/s step 0.25 (4601 points); FP64")
# FP64 flops per layer-evaluation (element assembly + one Schur step):
# 2*DFMA + DMUL + DADD executed per evaluated (layer, c) pair, from ncu
# instruction counters of the fused counting kernel's FP64 certificate on the
# 128-model case of this workload (23.07 M DFMA, 19.57 M DMUL, 3.70 M DADD over
# 460,800 layer-evaluations; profiles/). Every FP64 kernel runs the same
# element and Schur arithmetic. (The plain FP64 scan measured 162.3 before the
# exponential, rescaling and comparison changes.)
F_LAYER_FLOPS = 150.6
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
# DRAM bytes (read + write) of one count_certify launch (ncu, 128-model case:
# 527.1 KB read, 0 written): the exponential's 16 KB table once per launch,
# the rest (records and item tables) scaled by the models of a launch.
CERTIFY_DRAM_BYTES_FIXED = 2048 * 8
CERTIFY_DRAM_BYTES_PER_MODEL = (527.104e3 - CERTIFY_DRAM_BYTES_FIXED) / 128
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


def cpu_oracle_rate(models, grid, n_models: int, threads: int = 0, banded: bool = False):
    """Time the CPU oracle (dense LU), or with banded=True the CPU banded
    baseline (the paper's serial banded elimination restated), on the first
    n_models models of the workload, on `threads` host threads (0: all
    cores). Returns (curves/s, threads, sample description)."""
    import oracle
    oracle.build()
    cores = threads or os.cpu_count() or 1
    sub = models.subset(range(n_models))
    run = oracle.dispersion_banded if banded else oracle.dispersion
    t0 = time.perf_counter()
    run(sub.as_dict(), grid.c0, grid.dc, grid.n_c, n_threads=cores)
    dt = time.perf_counter() - t0
    return n_models / dt, cores, f"first {n_models} of the 1024 models, all 200 wavelengths, " \
                                 f"{dt:.1f} s on {cores} threads"


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    models, grid = W.uniform_batch()
    per_step = 16
    for _ in range(args.warmup):
        cpu_oracle_rate(models, grid, 4)
    times = []
    cores = os.cpu_count() or 1
    import oracle
    for s in range(args.steps):
        sub = models.subset(range((s * per_step) % 1024, (s * per_step) % 1024 + per_step))
        t0 = time.perf_counter()
        oracle.dispersion(sub.as_dict(), grid.c0, grid.dc, grid.n_c, n_threads=cores)
        times.append(time.perf_counter() - t0)
    value = per_step * args.steps / sum(times)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * float(np.mean(times)), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample_models_per_step": per_step},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{per_step} models x 200 wavelengths per step"},
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


def counting_evals(models, grid, idx, st, nlim, n32):
    """Per-item evaluations of the counting-search scan (plan precision 2).
    FP32 layer evaluations of the search: 1 + ceil(log3 npf) steps of two
    inertia counts for a located item, npf = grid points below the pole-free
    bound min_i beta_i sqrt(1 + (pi/(k h_i))^2). FP64 layer evaluations of
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
    steps = np.where(npf >= 2, 1 + np.ceil(np.log(np.maximum(npf, 2)) / np.log(3.0)), 1)
    search = np.where(npf >= 1, 2 * steps, 0)
    root = np.where(st == 0, idx.astype(np.int64), lim - 1)
    start = np.where(root >= npf, npf, 0)
    linear = np.where(counted, 0, np.maximum(root - start + 1, 0))
    live = lim >= 2
    e32 = int(np.sum(np.where(live, search + linear, 0) * nl))
    e64_counted = int(np.sum(np.where(live & counted, 2, 0) * nl))
    e64_fallback = int(np.sum(np.where(live & ~counted, 3, 0) * nl))
    return e32, e64_counted, e64_fallback, float(np.mean(counted))


def counting_roofline(models, grid, idx, st, nlim, n32, phases, peak64, micro, sms):
    """Roofline of the dominant kernel of a counting-search scan, the fused
    search + FP64 certificate: its FP64 work (2 layer-evaluation chains per
    counted item) against the FP64 pipe, from algorithmic layer evaluations /
    device time. Its FP32 search work runs on the FP32 pipe beside it and is
    reported separately."""
    e32, e64, e64_fb, frac_counted = counting_evals(models, grid, idx, st, nlim, n32)
    peak32 = FP32_FFMA_PER_CLK_SM * 2.0 * sms * SM_MAX_MHZ * 1e6
    t0 = phases[0] * 1e-3
    achieved = e64 * F_LAYER_FLOPS / t0
    return {"bound": "alu", "unit": "TFLOP/s",
            "achieved": achieved / 1e12, "peak": peak64 / 1e12, "frac": achieved / peak64,
            "traffic": CERTIFY_DRAM_BYTES_FIXED + CERTIFY_DRAM_BYTES_PER_MODEL * models.n_models,
            "kernel": "count_certify_kernel (FP64 pipe; FP32 search alongside)",
            "peak_source": "derived: 2 DFMA/clk/SM x 2 flop x SMs x 2070 MHz",
            "layer_evals_per_launch": e64, "flops_per_layer_eval": F_LAYER_FLOPS,
            "search_layer_evals_fp32": e32,
            "search_fp32_frac_of_fp32_peak": e32 * F_LAYER_FLOPS_FP32 / t0 / peak32,
            "fallback_check_layer_evals_fp64": e64_fb,
            "phases_ms": {"count_certify": phases[0], "fallback": phases[1],
                          "resolve64": phases[2]},
            "counted_fraction": frac_counted,
            "fp64_peak_microbenchmark": micro / 1e12}


def run_extras(args, masw, torch):
    """Secondary workloads on the same line: the ragged batch (autotuned
    persistent graph vs one launch per model), the differentiation batch
    (misfit + adjoint gradient per second) and the serving trace (p50/p99
    latency and curves/s of the continuous-batching server vs the plain
    one-request-at-a-time path, per arrival rate)."""
    from paper_2003_02256_gb300 import serving
    out = {}
    only = set(args.extras.split(",")) if args.extras else None

    def want(name):
        return only is None or name in only

    # ragged batch
    if want("ragged_batch"):
        out.update(extra_ragged(args, masw))
    if want("differentiation") or want("inversion"):
        out.update(extra_differentiation_inversion(masw, torch))
    if want("partition_study"):
        out.update(extra_partition_study(masw))
    if want("uniform_stress"):
        out.update(extra_uniform_stress(masw))
    if want("higher_modes"):
        out.update(extra_higher_modes(masw, torch))
    if want("leaky"):
        out.update(extra_leaky(masw, torch))
    if want("first_call"):
        out.update(extra_first_call(masw))
    if want("serving"):
        out.update(extra_serving(args, serving))
    return out


def extra_ragged(args, masw):
    out = {}
    m3, g3 = W.ragged_batch(n_models=args.ragged_models)
    with masw.Batch(m3, g3) as b:
        plan = b.autotune(reps=1)
        b.dispersion()
        times = []
        for _ in range(2):
            b.dispersion()
            times.append(b.last_scan_ms())
        t0 = time.perf_counter()
        b.dispersion(plain=True)
        plain_s = time.perf_counter() - t0
    out["ragged_batch"] = {
        "workload": f"{m3.n_models} models, N~U{{3..30}}, n_lambda~U{{30..400}} log-spaced to "
                    "2x total depth, 10% low-velocity layer; c grid 50..1200 step 0.25",
        "items": m3.n_items, "batched_curves_per_s": m3.n_models / (min(times) * 1e-3),
        "plain_curves_per_s": m3.n_models / plain_s, "plan": plan.as_dict()}
    return out


def extra_differentiation_inversion(masw, torch):
    out = {}
    # differentiation batch
    m4, g4, true = W.differentiation_batch()
    gold = np.loadtxt(os.path.join(ROOT, "tests", "golden", "differentiation_true_roots.txt"))
    ce = np.tile(W.noisy_observation(gold[:, 2], sigma=2.0), m4.n_models)
    with masw.Batch(m4, g4) as b:
        b.misfit_grad(ce)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        reps = 2
        for _ in range(reps):
            b.misfit_grad(ce)
        dt = (time.perf_counter() - t0) / reps
    out["differentiation"] = {"workload": "512 models x 12 layers, 150 wavelengths, LSQ misfit "
                                          "+ adjoint gradient (beta, h)",
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


def extra_partition_study(masw):
    out = {}
    # partition study (Section 3.2): per-wavelength work of Algorithm 1 on a
    # 40-wavelength decreasing curve, split over P ranks contiguously or modularly
    m1, g1 = W.single_curve()
    lam = sharding.variable_curve_wavelengths(40)
    var = W.Models(m1.n_layers, m1.h, m1.alpha, m1.beta, m1.rho,
                   np.array([lam.size], np.int32), lam)
    with masw.Batch(var, g1) as b:
        _, vidx, vst = b.dispersion()
    work = vidx.astype(np.float64) + 1.0
    out["partition_study"] = {
        "workload": "single-curve model, 40 log-spaced decreasing wavelengths 60..1 m, "
                    "work = determinants evaluated by Algorithm 1 (idx + 1)",
        "speedup": {str(P): {"modular": sharding.partition_speedup(work, P, "modular"),
                             "contiguous": sharding.partition_speedup(work, P, "contiguous")}
                    for P in (1, 2, 3, 4, 8, 16, 20, 24)},
        "paper_section_3_2": {"3": {"modular": 2.8, "contiguous": 1.9},
                              "8": {"modular": 7.0, "contiguous": 4.2}}}

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
    the host-output rate, an FP64 roofline of the continuation kernel: the
    layer-evaluations the linear scan needs for the items the batch scan
    leaves without a change (from one point below the scan limit to the
    change, or to the end of the grid) x F_LAYER_FLOPS, over the kernel's
    device time (CUDA events around the device-output call on the batch
    stream, less the batch scan's own event time)."""
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
    peak = FP64_DFMA_PER_CLK_SM * 2.0 * masw.sm_count() * SM_MAX_MHZ * 1e6 / 1e12
    out["leaky"] = {"workload": lm.meta["workload"] + ", host outputs",
                    "curves_per_s": lm.n_models / min(lms), "ms": 1e3 * min(lms),
                    "batch_scan_ms": float(np.median(lscan)),
                    "continuation_kernel_ms": k_ms,
                    "found_fraction": float(np.mean(lst == 0)),
                    "continued_fraction": float(np.mean(cont)),
                    "roofline": {"bound": "alu", "unit": "TFLOP/s", "achieved": achieved,
                                 "peak": peak, "frac": achieved / peak,
                                 "kernel": "leaky_scan64_kernel (FP64 pipe)",
                                 "layer_evals": evals, "flops_per_layer_eval": F_LAYER_FLOPS}}
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


def extra_serving(args, serving):
    out = {}
    # serving
    sampler = W.RandomWalkSampler()
    reqs = W.concat([sampler.next() for _ in range(args.serving_requests)])
    grid = W.Grid(50.0, 0.25, 4601)
    rates = {}
    for rate in (1e3, 3e3, 1e4, 3e4, 1e5, 1e6):
        arr = W.poisson_arrivals(reqs.n_models, rate=rate)
        with serving.Server(grid, max_slots=2048, chunks_per_tick=8,
                            mem_cap_bytes=16 << 30) as srv:
            lat, _, _, _, st = srv.run_trace(reqs, arr)
        with serving.Server(grid, max_slots=1, chunks_per_tick=1 << 20) as plain:
            lat_p, _, _, _, _ = plain.run_trace(reqs, arr)
        rates[f"{rate:g}"] = {"served": serving.latency_summary(lat, arr, reqs.n_models),
                              "plain": serving.latency_summary(lat_p, arr, reqs.n_models),
                              "ticks": st["ticks"], "max_in_flight": st["max_in_flight"]}
    out["serving"] = {"workload": f"{reqs.n_models} random-walk model evaluations per rate "
                                  "(layers 3..30, wavelengths 30..400), Poisson arrivals, "
                                  "16 GB admission cap", "rates_per_s": rates}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--extras", default=None,
                    help="comma-separated subset of the extras (ragged_batch, differentiation, "
                         "inversion, partition_study, uniform_stress, higher_modes, leaky, "
                         "first_call, serving); default all")
    ap.add_argument("--ragged-models", type=int, default=8192)
    ap.add_argument("--serving-requests", type=int, default=2000)
    ap.add_argument("--precision", type=int, default=None, choices=[0, 1, 2],
                    help="scan plan: 0 FP64 scan, 1 FP32 screen + FP64 decision, 2 counting "
                         "search + FP64 certificate (default: library)")
    ap.add_argument("--cpl", type=int, default=None, choices=[1, 2, 4],
                    help="scan plan test velocities per lane (2: paired FP32x2 screen)")
    ap.add_argument("--workload", default="uniform", choices=["uniform", "ragged"],
                    help="main workload (ragged only for profiling the ragged batch)")
    ap.add_argument("--models", type=int, default=1024,
                    help="models per GPU (smaller only for profiler captures)")
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
    stream = torch.cuda.current_stream()

    # weak scaling: the job's models are world x args.models seeded models; rank r
    # evaluates its contiguous shard (seeded per shard), no data-path collective
    if args.workload == "uniform":
        models, grid = W.uniform_batch(n_models=args.models, seed=W.SEED + 1000 * rank)
    else:
        models, grid = W.ragged_batch(n_models=args.models, seed=W.SEED + 3 + 1000 * rank)
    ce_host = W.noisy_observation(np.full(models.n_items, 250.0), sigma=30.0, seed=rank)
    batch = masw.Batch(models, grid)
    if args.precision is not None:
        batch.set_plan(precision=args.precision)
    if args.cpl is not None:
        batch.set_plan(cpl=args.cpl)
    if not args.no_autotune:
        plan = batch.autotune(reps=1)
    else:
        plan = batch.plan()

    # results of one pass (parity-checked in tests; used for the algorithmic count)
    ct, idx, st = batch.dispersion()
    nlim = np.array([int(np.sum(grid.c0 + np.arange(grid.n_c) * grid.dc < models.model(m)[2][-1]))
                     for m in range(models.n_models)])
    units = algorithmic_layer_evals(models, idx, st, nlim)
    executed = executed_layer_evals(models, idx, st, nlim, plan.cpl)

    ce = torch.from_numpy(ce_host).cuda()
    phi = torch.empty(models.n_models, dtype=torch.float64, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def step():
        masw.misfit(batch.handle, ce, masw.MISFIT_LSQ, 2.0, phi)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    scan_ms = []
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record(stream)
            step()
            ev[k][1].record(stream)
            torch.cuda.synchronize()
            scan_ms.append(batch.last_scan_ms())
        torch.cuda.synchronize()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = float(np.sum(step_ms))
    total_ms = sharding.max_over_ranks(total_ms, device="cuda")
    value = world * models.n_models * args.steps / (total_ms * 1e-3)

    # plain one-curve-per-launch path (same kernel body, one launch + sync per model)
    plain_ms = []
    for _ in range(0 if args.no_plain else 2):
        t0 = time.perf_counter()
        batch.dispersion(plain=True)
        plain_ms.append(1e3 * (time.perf_counter() - t0))
    plain_value = models.n_models / (min(plain_ms) * 1e-3) if plain_ms else None

    # end to end through the C ABI with host buffers: upload of the step's
    # model parameters and C_e from pinned memory, misfit read back to host
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    hh, ha, hb, hr, hce = (pin(x) for x in (models.h, models.alpha, models.beta, models.rho, ce_host))
    hphi = torch.empty(models.n_models, dtype=torch.float64).pin_memory()
    e2e_ms = []
    for k in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        masw.model_batch_update(batch.handle, hh, ha, hb, hr)
        masw.misfit(batch.handle, hce, masw.MISFIT_LSQ, 2.0, hphi)
        torch.cuda.synchronize()
        if k >= args.warmup:
            e2e_ms.append(1e3 * (time.perf_counter() - t0))
    e2e_total = float(np.sum(e2e_ms))
    e2e_total = sharding.max_over_ranks(e2e_total, device="cuda")
    e2e_value = world * models.n_models * args.steps / (e2e_total * 1e-3)
    h2d = sum(x.numel() * 8 for x in (hh, ha, hb, hr, hce))
    d2h = hphi.numel() * 8

    # per-kernel device times of the two-precision scan (same kernels, launched
    # without the graph so events can sit between them)
    phases = None
    unresolved = None
    fallback = None
    n32 = None
    if plan.precision >= 1:
        batch.set_plan(use_graph=0)
        ph = []
        for _ in range(3):
            flush.zero_()
            batch.dispersion()
            ph.append(masw.last_scan_phases(batch.handle))
        unresolved = batch.last_scan_unresolved()
        fallback = batch.last_scan_fallback()
        n32 = np.empty(models.n_items, dtype=np.int32)
        masw.last_scan_screen(batch.handle, n32)
        batch.set_plan(use_graph=plan.use_graph)
        phases = [float(np.mean([p[i] for p in ph])) for i in range(3)]

    # roofline of the scan kernel: algorithmic FP64 flops / device time, against
    # the FP64 peak derived from unit counts and the maximum SM clock
    # (2 DFMA per clock per SM x 2 flops x SMs x 2070 MHz); the live DFMA
    # microbenchmark is reported beside it
    micro = masw.fp64_peak()
    peak = FP64_DFMA_PER_CLK_SM * 2.0 * masw.sm_count() * SM_MAX_MHZ * 1e6
    scan_avg = float(np.mean(scan_ms)) * 1e-3
    if phases is None:
        achieved = units * F_LAYER_FLOPS / scan_avg
        roofline = {"bound": "alu", "achieved": achieved / 1e12, "peak": peak / 1e12,
                    "unit": "TFLOP/s", "frac": achieved / peak,
                    "traffic": SCAN_DRAM_BYTES_PER_MODEL * models.n_models,
                    "kernel": "scan_kernel (FP64 pipe)",
                    "peak_source": "derived: 2 DFMA/clk/SM x 2 flop x SMs x 2070 MHz",
                    "peak_microbenchmark": micro / 1e12,
                    "layer_evals_per_launch": units, "flops_per_layer_eval": F_LAYER_FLOPS,
                    "executed_layer_evals_per_launch": executed,
                    "scan_ms": scan_avg * 1e3}
    elif plan.precision == 2:
        roofline = counting_roofline(models, grid, idx, st, nlim, n32, phases, peak, micro,
                                     masw.sm_count())
        roofline.update({"scan_ms": scan_avg * 1e3, "unresolved_items": unresolved,
                         "fallback_items": fallback})
    else:
        peak32 = FP32_FFMA_PER_CLK_SM * 2.0 * masw.sm_count() * SM_MAX_MHZ * 1e6
        t_screen = phases[0] * 1e-3
        achieved = units * F_LAYER_FLOPS_FP32 / t_screen
        roofline = {"bound": "alu", "achieved": achieved / 1e12, "peak": peak32 / 1e12,
                    "unit": "TFLOP/s", "frac": achieved / peak32,
                    "traffic": SCREEN_DRAM_BYTES_PER_MODEL * models.n_models,
                    "kernel": "screen32_kernel (FP32 pipe)",
                    "peak_source": "derived: 128 FFMA/clk/SM x 2 flop x SMs x 2070 MHz",
                    "layer_evals_per_launch": units,
                    "flops_per_layer_eval": F_LAYER_FLOPS_FP32,
                    "executed_layer_evals_per_launch": executed,
                    "scan_ms": scan_avg * 1e3,
                    "phases_ms": {"screen32": phases[0], "verify64": phases[1],
                                  "resolve64": phases[2]},
                    "fp64_peak_derived": peak / 1e12, "fp64_peak_microbenchmark": micro / 1e12,
                    "unresolved_items": unresolved}

    extras = None
    if rank == 0 and world == 1 and not args.no_extras:
        extras = run_extras(args, masw, torch)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, cores, sample = cpu_oracle_rate(models, grid, min(256, models.n_models))
        v1, _, sample1 = cpu_oracle_rate(models, grid, min(8, models.n_models), threads=1)
        vb, _, sample_b = cpu_oracle_rate(models, grid, min(512, models.n_models), banded=True)
        vb1, _, sample_b1 = cpu_oracle_rate(models, grid, min(16, models.n_models), threads=1,
                                            banded=True)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
               "single_thread": {"value": v1, "unit": UNIT, "sample": sample1},
               "banded": {"value": vb, "unit": UNIT, "cores": cores,
                          "kind": "CPU banded elimination (the paper's serial C, sparse variant, "
                                  "restated; pinned to the oracle)",
                          "sample": sample_b,
                          "single_thread": {"value": vb1, "unit": UNIT, "sample": sample_b1}}}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": WORKLOAD, "models_per_gpu": models.n_models,
                           "items_per_gpu": models.n_items, "seed": W.SEED,
                           "l2": "flushed between timed steps (256 MB write)",
                           "step": "Algorithm 1 scan of every item + Algorithm 2 misfit",
                           "plan": plan.as_dict(), "parallelism": f"replicas x{world}"},
                "clocks": clk.summary(),
                "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                        "d2h_bytes_per_step": d2h},
                # per step: the scan's kernels (precision 0: scan; 1: screen, check,
                # mode-count search, re-scan; 2: counting search + certificate,
                # fallback scan, check, mode-count search, re-scan) and the misfit
                "gpu_launches": {0: 2, 1: 5, 2: 6}[plan.precision] * args.steps,
                "roofline": roofline,
                "cpu_baseline": cpu,
                "plain_gpu": None if plain_value is None else {
                    "value": plain_value, "unit": UNIT, "ms_per_step": min(plain_ms),
                    "speedup_of_batched": value / world / plain_value},
                "found_fraction": float(np.mean(st == 0)),
                "extras": extras}
        print(json.dumps(line), flush=True)
    batch.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
