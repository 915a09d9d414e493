#!/usr/bin/env python
"""Benchmark of one VEGAS iteration on GB300 (sm_103a) through the C ABI.

Workload (one step = one Vegas iteration, sampling + finalize + refine, of two
integrals, 2e7 samples in all):
  * d = 8 symmetric Gaussian f = (a sqrt(pi))^-8 exp(-sum (x - 1/2)^2/a^2), a = 0.1
  * d = 8 Genz oscillatory f = cos(2 pi 0.3 + sum c_i x_i), c_i ~ U(0, 1), seed 1
  * 50 bins per dimension, 1e7 samples per iteration each, alpha = 1.5,
  * FP32 sampling / grid map / integrand, FP64 accumulators (VEGAS_FP32_ACC64).
The paper's own workload (the single-top LO integrand, Sec. 3.1) is not
available; these seeded synthetic integrands stand in for it.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle instead, on the host cores, on a bounded sample of the same workload.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Vegas samples/s (% of roofline)"
UNIT = "samples/s"
D, NBINS, NEVENTS, ALPHA = 8, 50, 10_000_000, 1.5
PRECISION = "fp32_acc64"
PROFILE_EVERY = 4             # timed steps per step with kernel events
WORKLOAD = "d=8 Gaussian a=0.1 + d=8 Genz oscillatory (c~U(0,1) seed 1), 50 bins, 1e7 samples/iter each"

# The workload's identity, the same in both arms (the arithmetic is in "dtype").
CONFIG = {"workload": WORKLOAD, "integrals": 2, "dims": D, "bins": NBINS, "samples_per_iteration": NEVENTS}

# Serving sweep: Poisson arrival rates and requests per rate (about two
# seconds of arrivals each, at most 1e4: 1e4 requests at 10/s would arrive
# over 1000 s).
SERVING_RATES = (10.0, 100.0, 1000.0, 10000.0)


def serving_requests(rate: float) -> int:
    return int(min(10_000, max(20, round(2.0 * rate))))

# Unit counts used for the issue roofline (per SM per clock); the measured
# costs come from paper_2010_09341_gb300/calib/pipe_costs.cu.
ISSUE_PER_SM_CLK = 128.0      # 4 schedulers x 32 lanes: one warp instruction each per clock
MUFU_PER_SM_CLK = 32.0        # special-function lanes (ex2.approx measured at 4 cycles/warp/scheduler)
MULWIDE_ISSUE_CYCLES = 4.0    # a 32x32->64 multiply holds its scheduler for 4 cycles (measured 4.05)
FP64_TFLOPS_NOMINAL = 1.25    # GB300 dense FP64 (FMA = 2 flop); measured DFMA rate gives 1.06


def _integrals():
    from paper_2010_09341_gb300 import workloads as W
    return [("gauss_sym", W.gauss_sym_params(0.1)), ("genz_osc", W.genz_osc_params(D, seed=1))]


def ctypes_sizeof_result() -> int:
    """Bytes of one combined result read back (vegas_result_t)."""
    import ctypes
    from paper_2010_09341_gb300 import _native as nat
    return ctypes.sizeof(nat.VegasResult)


# ------------------------------------------------------------- op counting
def ops_per_sample(family: str, d: int, precision: str):
    """Algorithmic operations of one sample, by pipe (thread-level counts).

    Philox4x32-10: 10 rounds x (2 wide multiplies + 2 three-input xors) per
    4 words (round keys are per-thread constants).  Per dimension: 1 wide
    multiply (bin split), 1 conversion of the in-bin position, 1 cell index,
    1 table address, 1 table load, 1 FMA (x), 1 multiply (J), 1 histogram
    address, 1 shared integer atomic, plus the integrand's per-dimension ops
    (a family that takes x about a centre gets it from the table: the
    symmetric Gaussian's (x - 1/2)^2 is one FMA); J *= N^4 once per 4
    dimensions.  Per sample: integrand finish, v = J f, v^2, non-finite test
    (2), the fixed-point histogram value (scale, convert, clamp, range test:
    5), the two sums (FP32 partials + FP64 flush: 2 adds, 2 for the chunk
    bookkeeping and 4 FP64 ops per 16 samples; Kahan: 8 FP32 ops), loop (3).
    Wide multiplies (32x32->64) also count on their own pipe: 20 per Philox
    call plus one per dimension.  The FP64 path: fp64_ops_per_sample.
    """
    per_dim_f = {"gauss_sym": 1, "genz_osc": 1, "genz_gauss": 2, "genz_prod": 3,
                 "genz_corner": 1, "sum": 1, "const": 0, "lo": 0, "lo_pdf": 0}[family]
    finish = {"gauss_sym": 2, "genz_osc": 6, "genz_gauss": 2, "genz_prod": 1,
              "genz_corner": 3, "sum": 0, "const": 0, "lo": 20, "lo_pdf": LO_PDF_FINISH}[family]
    mufu = {"gauss_sym": 1, "genz_osc": 1, "genz_gauss": 1, "genz_prod": 1,
            "genz_corner": 2, "sum": 0, "const": 0, "lo": 2, "lo_pdf": 4}[family]
    calls = math.ceil(d / 4)
    philox = 40 * calls
    per_dim = (9 + per_dim_f) * d + d // 4
    fp64 = 0
    hist = 5
    if precision == "fp32_kahan":
        acc = 8
    elif precision == "fp32_acc64":
        acc = 4 + 0.25
        fp64 = 0.25
    else:
        acc = 3
        hist = 0
        fp64 = fp64_ops_per_sample(family, d)
    total = philox + per_dim + finish + 2 + 2 + hist + acc + 3
    return {"total": total, "fp64": fp64, "mufu": mufu, "mulwide": 20 * calls + d}


# The LO toy on a density grid (F_LO_PDF), FP32, per sample after the map:
# the LO kinematics, cuts, Breit-Wigner and angular factor (20, as the LO
# family, its power law replaced by the two densities); three grid coordinates
# (log2 on the MUFU, subtract, scale, clamp (2), truncate, cap, convert back,
# fraction: 9 each); three sets of cubic weights (13 each); two bicubic
# lookups of 4 x 4 knots (16 shared-memory loads, 20 FMAs, 3 for the address:
# 39 each); and the product of the two densities (2).
LO_PDF_FINISH = 20 + 3 * 9 + 3 * 13 + 2 * 39 + 2


def strat_ops_per_sample(family: str, d: int, precision: str, P: int):
    """ops_per_sample for the stratified hybrid with P samples per hypercube:
    per dimension the stratum word (a funnel shift, and the hypercube's bits
    shifted once per hypercube); per sample the deviation from the hypercube's
    first value and its two running sums (3); per hypercube the spread
    b - a^2 / P clipped at 0 and added (4), the hypercube index and first
    sample index (2) and its loop (3)."""
    o = dict(ops_per_sample(family, d, precision))
    o["total"] += d * (1 + 1 / P) + 3 + (4 + 2 + 3) / P
    return o


# Cost of one call of an FP64 function in DFMA issue slots of the FP64 pipe:
# its measured cycles per warp instruction over a DFMA's (76), from
# paper_2010_09341_gb300/calib/pipe_costs.cu on one GB300.  exp2 is the
# library's own table-driven 2^x (vegas::fexp2, 9 FP64 operations; CUDA's
# exp2 costs 17.0), the others CUDA's functions.
FP64_CALL_DFMA = {"exp2": 9.9, "cos": 17.5, "log2": 30.4, "rcp": 4.7}


def fp64_ops_per_sample(family: str, d: int) -> float:
    """FP64-pipe operations of one sample of the FP64 path (VEGAS_FP64): per
    dimension the map FMA, the Jacobian multiply and the histogram add (the
    shared FP64 atomic's add), plus the integrand's per-dimension ops; per
    sample v = J f, v^2 and the sums of v and v^2 (4), and the integrand's
    finish, library calls at their measured DFMA-equivalent cost."""
    per_dim_f = {"gauss_sym": 1, "genz_osc": 1, "genz_gauss": 2, "genz_prod": 3,
                 "genz_corner": 1, "sum": 1, "const": 0, "lo": 0}[family]
    c = FP64_CALL_DFMA
    finish = {"gauss_sym": 1 + c["exp2"], "genz_osc": c["cos"], "genz_gauss": 1 + c["exp2"],
              "genz_prod": c["rcp"], "genz_corner": 1 + c["log2"] + c["exp2"], "sum": 0, "const": 0,
              "lo": 14 + 2 * c["rcp"]}[family]
    return (3 + per_dim_f) * d + 4 + finish


def roofline_samples_per_s(ops, sms: int, clk_hz: float) -> dict:
    """Bounds in samples/s from the per-sample operation counts.

    "issue": every operation costs one issue slot of a scheduler (4 per SM,
    32 lanes each), except a 32x32->64 multiply, which occupies its
    scheduler for 4 cycles and issues nothing else meanwhile (measured:
    mul.hi 4.05 cycles per warp instruction; a multiply-and-xor chain
    interleaved with two independent FMAs takes the sum of the two times).
    Half-rate integer operations (three-input logic, 32-bit multiply-add:
    2 cycles measured) are charged one slot, so the bound is optimistic for
    them.  The other pipes bound separately: FP64 at the nominal 1.25
    TFLOP/s (2 FMA lanes/clk/SM), MUFU 32 lanes/clk/SM.
    """
    fp64_per_sm_clk = FP64_TFLOPS_NOMINAL * 1e12 / 2.0 / (sms * clk_hz)
    cycles = (ops["total"] - ops.get("mulwide", 0)) + MULWIDE_ISSUE_CYCLES * ops.get("mulwide", 0)
    bounds = {"issue": sms * clk_hz * ISSUE_PER_SM_CLK / cycles}
    if ops["fp64"]:
        bounds["fp64"] = sms * clk_hz * fp64_per_sm_clk / ops["fp64"]
    if ops["mufu"]:
        bounds["mufu"] = sms * clk_hz * MUFU_PER_SM_CLK / ops["mufu"]
    return bounds


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self._t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------- reference arm
def oracle_rate(threads: int, seconds: float = 0.3):
    """Calibration: oracle samples/s on ``threads`` host threads."""
    import oracle as O
    e = O.uniform_edges(D, NBINS)
    n = 5_000 * threads
    done = 0
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < seconds:
        for fam, p in _integrals():
            O.iterate(D, NBINS, e, fam, p, 0, 1, 0, n, threads=threads)
            done += n
    return done / (time.perf_counter() - t0)


def oracle_samples_per_s(seconds: float, threads: int, rate=None, t=0):
    """Time the FP64 oracle on host threads over a bounded sample of the
    workload (both integrals, iteration t, uniform grid), about ``seconds``."""
    import oracle as O
    e = O.uniform_edges(D, NBINS)
    if rate is None:
        rate = oracle_rate(threads)
    n = max(threads * 100, int(rate * seconds / 2))
    t0 = time.perf_counter()
    for k, (fam, p) in enumerate(_integrals()):
        O.iterate(D, NBINS, e, fam, p, 0, k, t, n, threads=threads)
    dt = time.perf_counter() - t0
    return 2 * n / dt, 2 * n, dt


def run_reference(args):
    """The oracle as it stands, timed on this host's cores: each step a
    bounded sample of the workload, the whole run sized to a few minutes."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    threads = os.cpu_count() or 1
    rate = oracle_rate(threads)
    per_step_s = min(args.ref_seconds, 120.0 / max(1, args.steps + args.warmup))
    for w in range(args.warmup):
        oracle_samples_per_s(per_step_s, threads, rate, t=w)
    per_step = []
    n_total = 0
    for k in range(args.steps):
        _, n, dt = oracle_samples_per_s(per_step_s, threads, rate, t=k)
        per_step.append(dt)
        n_total += n
    value = n_total / sum(per_step)
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * sum(per_step) / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(CONFIG, parallelism="host threads (%d)" % threads),
        "method": {"step": "each step: %d samples per integral of iteration t on the uniform grid"
                   % (n_total // (2 * args.steps))},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": "%d samples over %d steps (%.1f s)"
                         % (n_total, args.steps, sum(per_step))},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out))
    return 0


# ------------------------------------------------------ other workloads
def _time_single(V, torch, family, params, d, N, n, prec, iters, warm=2, iid=0):
    """samples/s of `iters` iterations (sample + finalize + refine) of one
    integral, after `warm` untimed ones; device time with CUDA events."""
    cfg = V.Config(n_dim=d, n_events=n, n_bins=N, alpha=ALPHA, seed=0, integral_id=iid,
                   precision=prec)
    ctx = V.vegas_create(cfg, family, params)
    for _ in range(warm):
        V.vegas_step(ctx, sync=False)
    V.vegas_profile(ctx, True)
    s = torch.cuda.current_stream()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(s)
    for _ in range(iters):
        V.vegas_step(ctx, sync=False)
    b.record(s)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    kms = V.vegas_profile_read(ctx)
    res = V.vegas_result(ctx)
    V.vegas_destroy(ctx)
    k_ms = sum(kms) / max(1, len(kms))
    out = {"samples_per_s": n * iters / (ms / 1e3), "ms_per_iter": ms / iters,
           "kernel_ms": k_ms, "I": res["I"], "sigma": res["sigma"]}
    # the sampling kernel against the tightest bound of its family, d and
    # precision: instruction issue in the FP32 modes, the FP64 pipe in FP64
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    bounds = roofline_samples_per_s(ops_per_sample(family, d, prec), sms, 2070e6)
    pipe = min(bounds, key=bounds.get)
    out["roofline"] = {"bound": "alu" if pipe == "issue" else pipe, "pipe": pipe,
                       "roofline_samples_per_s": bounds[pipe], "frac": (n / (k_ms / 1e3)) / bounds[pipe]}
    if prec == "fp64":
        out["roofline"]["fp64_ops_per_sample"] = fp64_ops_per_sample(family, d)
    return out


def _time_strat(V, torch, family, params, d, N, n, prec, iters=10, warm=5):
    """Plain against stratified sampling (vegas_set_strata(-1)) on one integral:
    kernel time per iteration, the standard error of an iteration times the
    square root of its samples (sigma sqrt(n), the per-sample spread the
    estimator sees), and the time to reach a given sigma relative to plain
    sampling (sigma^2 t, lower is better)."""
    out = {}
    for B in (0, -1):
        cfg = V.Config(n_dim=d, n_events=n, n_bins=N, alpha=ALPHA, seed=0, integral_id=0,
                       precision=prec)
        ctx = V.vegas_create(cfg, family, params)
        V.vegas_set_strata(ctx, B)
        for _ in range(warm):
            V.vegas_step(ctx, sync=False)
        V.vegas_profile(ctx, True)
        sig = []
        for _ in range(iters):
            sig.append(V.vegas_step(ctx)[1])
        kms = V.vegas_profile_read(ctx)
        Bt, P, used = V.vegas_get_strata(ctx)
        res = V.vegas_result(ctx)
        V.vegas_destroy(ctx)
        k_ms = sum(kms) / len(kms)
        s_rms = math.sqrt(sum(x * x for x in sig) / len(sig))
        sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
        ops = strat_ops_per_sample(family, d, prec, P) if P else ops_per_sample(family, d, prec)
        bounds = roofline_samples_per_s(ops, sms, 2070e6)
        pipe = min(bounds, key=bounds.get)
        out["stratified" if B else "plain"] = {
            "hypercubes": 2 ** Bt if P else 0, "samples_per_hypercube": P, "samples": used,
            "kernel_ms": k_ms, "samples_per_s": used / (k_ms / 1e3),
            "sigma_sqrt_n": s_rms * math.sqrt(used), "I": res["I"], "sigma": res["sigma"],
            "roofline": {"bound": "alu" if pipe == "issue" else pipe, "pipe": pipe,
                         "ops_per_sample": ops["total"], "roofline_samples_per_s": bounds[pipe],
                         "frac": (used / (k_ms / 1e3)) / bounds[pipe]}}
    a, b = out["plain"], out["stratified"]
    out["time_to_equal_sigma_vs_plain"] = (b["sigma_sqrt_n"] ** 2 / b["samples_per_s"]) / \
        (a["sigma_sqrt_n"] ** 2 / a["samples_per_s"])
    return out


USER_GENZ_GAUSS = r"""
template <class T> __device__ T user_integrand(const T *x, int d, const T *p) {
    T q = T(0);
    for (int j = 0; j < d; ++j) {
        const T t = p[j] * (x[j] - p[d + j]);
        q += t * t;
    }
    return exp(-q);
}
"""


def _time_user(V, torch, d=8, N=NBINS, n=NEVENTS, prec=PRECISION, iters=10, warm=3):
    """A user integrand compiled at run time (the Genz Gaussian as user source,
    d = 8, c ~ U(0.5, 5), w ~ U(0, 1), seed 2) against the same integrand as the
    built-in family: run-time compilation time and kernel time per iteration."""
    from paper_2010_09341_gb300 import workloads as W
    p = W.genz_params("genz_gauss", d, seed=2)
    out = {}
    for kind in ("user", "builtin"):
        cfg = V.Config(n_dim=d, n_events=n, n_bins=N, alpha=ALPHA, seed=0, integral_id=0,
                       precision=prec)
        t0 = time.perf_counter()
        if kind == "user":
            ctx = V.vegas_create(cfg, "user", p, source=USER_GENZ_GAUSS + "\n// %d\n" % os.getpid())
        else:
            ctx = V.vegas_create(cfg, "genz_gauss", p)
        t_create = time.perf_counter() - t0
        for _ in range(warm):
            V.vegas_step(ctx, sync=False)
        V.vegas_profile(ctx, True)
        for _ in range(iters):
            V.vegas_step(ctx, sync=False)
        kms = V.vegas_profile_read(ctx)
        res = V.vegas_result(ctx)
        V.vegas_destroy(ctx)
        k_ms = sum(kms) / len(kms)
        out[kind] = {"create_s": t_create, "kernel_ms": k_ms, "samples_per_s": n / (k_ms / 1e3),
                     "I": res["I"], "sigma": res["sigma"]}
    # both against the built-in family's counted operations (the algorithmic
    # work of this integrand; the user source also subtracts the centre and
    # scales x per dimension)
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    bounds = roofline_samples_per_s(ops_per_sample("genz_gauss", d, prec), sms, 2070e6)
    pipe = min(bounds, key=bounds.get)
    for kind in ("user", "builtin"):
        out[kind]["roofline"] = {"bound": "alu" if pipe == "issue" else pipe, "pipe": pipe,
                                 "roofline_samples_per_s": bounds[pipe],
                                 "frac": out[kind]["samples_per_s"] / bounds[pipe],
                                 "basis": "the built-in Genz Gaussian's counted operations"}
    out["workload"] = "Genz Gaussian d=%d, %d bins, %g samples/iter, %s; user source vs built-in family" % (
        d, N, n, prec)
    return out


def _time_lo_pdf(V, torch, n=100_000_000, iters=10, warm=2, prec="fp32_kahan"):
    """Config 3 with the density taken from a grid (96 x 48 knots of a synthetic
    scale-dependent density, bicubic in ln x, ln Q^2 at Q^2 = shat) against the
    analytic LO toy: samples/s of the sampling kernel and of whole iterations."""
    from paper_2010_09341_gb300 import workloads as W
    xg, u0, u1, v0, v1 = W.pdf_grid(96, 48)
    t = torch.from_numpy(xg).cuda()
    cfg = V.Config(n_dim=3, n_events=n, n_bins=100, alpha=ALPHA, seed=0, integral_id=0, precision=prec)
    ctx = V.vegas_create(cfg, "lo_pdf", W.lo_params())
    V.vegas_set_pdf_grid(ctx, t, u0, u1, v0, v1)
    for _ in range(warm):
        V.vegas_step(ctx, sync=False)
    V.vegas_profile(ctx, True)
    s = torch.cuda.current_stream()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(s)
    for _ in range(iters):
        V.vegas_step(ctx, sync=False)
    b.record(s)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    kms = V.vegas_profile_read(ctx)
    res = V.vegas_result(ctx)
    V.vegas_destroy(ctx)
    k_ms = sum(kms) / len(kms)
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    ops = ops_per_sample("lo_pdf", 3, prec)
    bounds = roofline_samples_per_s(ops, sms, 2070e6)
    pipe = min(bounds, key=bounds.get)
    return {"workload": "LO toy d=3, density from a 96x48 (ln x, ln Q^2) grid at Q^2 = shat, 100 bins, "
                        "%g samples/iter, %s" % (n, prec),
            "samples_per_s": n * iters / (ms / 1e3), "kernel_ms": k_ms,
            "kernel_samples_per_s": n / (k_ms / 1e3), "ms_per_iter": ms / iters,
            "I": res["I"], "sigma": res["sigma"],
            "roofline": {"bound": "alu" if pipe == "issue" else pipe, "pipe": pipe, "ops_per_sample": ops["total"],
                         "roofline_samples_per_s": bounds[pipe], "frac": (n / (k_ms / 1e3)) / bounds[pipe]}}


def _time_batched(V, torch, steps=8, warm=2):
    """The uneven 512-integral mix: one step = one iteration of every integral."""
    from paper_2010_09341_gb300 import workloads as W
    mix = W.batch_mix(512, seed=2)
    b = V.Batch(max_slots=512, pool_bytes=256 << 20, precision="fp32_kahan")
    for it in mix:
        b.add(V.Config(n_dim=it.d, n_events=it.n_events, n_bins=it.n_bins, alpha=ALPHA, seed=0,
                       integral_id=it.integral_id, precision="fp32_kahan"), it.family, it.params)
    for _ in range(warm):
        b.step()
        b.wait()
    # launch shapes: tile samples x threads per block x shared-memory layout
    cands = [(t, th, lay) for t in (65536, 131072, 262144, 524288) for th in (512, 640, 768)
             for lay in (1, 2)]
    import tempfile
    cache = os.path.join(tempfile.mkdtemp(prefix="vegas_tune_"), "tune.json")
    shape, ms = b.autotune_shapes(cands, reps=2, cache=cache)
    b.step()
    b.wait()
    t0 = time.perf_counter()
    for _ in range(steps):
        b.step()
        b.wait()
    dt = time.perf_counter() - t0
    n_total = sum(it.n_events for it in mix)
    b.close()
    # issue roofline of one step: every integral's samples at its own bound
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    roof_s = 0.0
    for it in mix:
        bounds = roofline_samples_per_s(ops_per_sample(it.family, it.d, "fp32_kahan"), sms, 2070e6)
        roof_s += it.n_events / min(bounds.values())
    ms_step = 1e3 * dt / steps
    return {"workload": "512 integrals, d ~ U{2..16}, Genz gauss/prod/corner, c ~ U(0.5,5), "
                        "n ~ logU(1e4,1e7) per iteration, 50 bins, FP32 Kahan, seed 2",
            "samples_per_step": n_total, "steps": steps, "ms_per_step": ms_step,
            "roofline": {"bound": "alu", "roofline_ms_per_step": 1e3 * roof_s,
                         "roofline_samples_per_s": n_total / roof_s,
                         "frac": 1e3 * roof_s / ms_step,
                         "basis": "sum over the 512 integrals of n / (issue bound of its family and d) "
                                  "at %d SMs x 2070 MHz; the step time includes finalize, refinement "
                                  "and the graph's plan upload and result download" % sms},
            "samples_per_s": n_total * steps / dt,
            "integral_iterations_per_s": 512 * steps / dt,
            "shape": shape, "tile_samples": shape["tile_samples"],
            "autotune_ms": {"%d/%d/%d" % c: round(m, 4) for c, m in zip(cands, ms) if m >= 0},
            "timing": "wall clock per step incl. graph launch and result download"}


def _served_roofline(reqs, wall_s, prec="fp32_kahan"):
    """The served work at the issue bound: the sum over completed requests of
    their samples over the bound of their family and dimension, against the
    wall time (a load figure below saturation, where arrivals leave the GPU
    idle; the kernel's efficiency on the served mix at saturation)."""
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    roof_s = 0.0
    for r in reqs:
        if r.done >= 0 and r.result:
            b = roofline_samples_per_s(ops_per_sample(r.family, r.d, prec), sms, 2070e6)
            roof_s += r.result["samples"] / min(b.values())
    return {"bound": "alu", "roofline_s": roof_s, "frac_of_wall": roof_s / wall_s if wall_s > 0 else None,
            "basis": "sum over completed requests of samples / issue bound of (family, d) at %d SMs x 2070 MHz"
                     % sms}


def _serving_compare(V, rate, n_requests, target, budget):
    """The same Poisson request stream through the batched FP32-Kahan server
    and through the plain FP64 single-integral form (one context at a time),
    both with real-time arrivals and the same sample schedule and stopping
    rules: integrals/s and latency of each."""
    from paper_2010_09341_gb300 import serve as S
    from paper_2010_09341_gb300 import workloads as W
    stream = W.request_stream(rate=rate, n_requests=n_requests, seed=3)
    srv = S.Server(max_slots=1024, pool_bytes=512 << 20)
    st32 = srv.run(S.requests_from(stream, budget=budget, target=target), realtime=True, time_limit=120)
    srv.batch.close()
    st64 = S.serve_single_fp64(S.requests_from(stream, budget=budget, target=target), time_limit=120)
    return {"rate_per_s": rate, "requests": n_requests, "target_rel": target, "budget": budget,
            "arrival": "Poisson, real time, the same stream for both",
            "batched_fp32_kahan": st32, "fp64_single": st64,
            "integrals_per_s_ratio": (st32["integrals_per_s"] / st64["integrals_per_s"]
                                      if st64["integrals_per_s"] else None),
            "converged_per_s_ratio": (st32["converged_per_s"] / st64["converged_per_s"]
                                      if st64["converged_per_s"] else None)}


def _serving(V, rate, n_requests, target, budget, fp64_sample=0):
    from paper_2010_09341_gb300 import serve as S
    from paper_2010_09341_gb300 import workloads as W
    stream = W.request_stream(rate=rate, n_requests=n_requests, seed=3)
    reqs = S.requests_from(stream, budget=budget, target=target)
    srv = S.Server(max_slots=1024, pool_bytes=512 << 20)
    st = srv.run(reqs, realtime=True, time_limit=120)
    srv.batch.close()
    out = {"rate_per_s": rate, "target_rel": target, "budget": budget, **st}
    out["roofline"] = _served_roofline(reqs, st["wall_s"])
    if fp64_sample:
        # the same first requests, all queued at t = 0, through both forms
        def queued():
            sub = S.requests_from(stream[:fp64_sample], budget=budget, target=target)
            for r in sub:
                r.arrival = 0.0
            return sub
        srv = S.Server(max_slots=1024, pool_bytes=512 << 20)
        st32 = srv.run(queued(), realtime=False, time_limit=120)
        srv.batch.close()
        st64 = S.serve_single_fp64(queued(), time_limit=120)
        out["same_requests"] = {
            "requests": fp64_sample, "arrival": "all queued at t = 0",
            "batched_fp32_kahan": st32, "fp64_single": st64,
            "integrals_per_s_ratio": (st32["integrals_per_s"] / st64["integrals_per_s"]
                                      if st64["integrals_per_s"] else None),
            "converged_per_s_ratio": (st32["converged_per_s"] / st64["converged_per_s"]
                                      if st64["converged_per_s"] else None)}
    return out


def _traffic_from_profile():
    """DRAM bytes per sampling-kernel launch from the committed ncu summary,
    if the kernel sources still hash to what was profiled; else None."""
    import hashlib
    import re
    prof = os.path.join(ROOT, "profiles", "sample_kernel_d8_gauss.md")
    src = os.path.join(ROOT, "paper_2010_09341_gb300", "csrc")
    try:
        txt = open(prof).read()
        h = hashlib.sha256()
        for f in ("vegas_device.cuh", "vegas_sample.cuh"):
            h.update(open(os.path.join(src, f), "rb").read())
        want = re.search(r"kernel_source_sha256:\s*([0-9a-f]{64})", txt).group(1)
        if want != h.hexdigest():
            return None
        return float(re.search(r"traffic_bytes_per_launch:\s*([0-9.]+)", txt).group(1))
    except (OSError, AttributeError):
        return None


# ----------------------------------------------------------------- GPU arm
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=200)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--ref-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the other workloads")
    ap.add_argument("--only", choices=["batched", "serving", "lo", "config1", "fp64", "strat", "user", "lo_pdf"],
                    default=None,
                    help="run just one of the other workloads and print its JSON (for profiling)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    assert args.warmup >= 3, "at least 3 warm-up steps"

    import numpy as np
    import torch
    import torch.distributed as dist

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if args.only:
        from paper_2010_09341_gb300 import build as B
        from paper_2010_09341_gb300 import vegas as V
        from paper_2010_09341_gb300 import workloads as W
        B.build()
        if args.only == "batched":
            out = _time_batched(V, torch, steps=args.steps, warm=args.warmup)
        elif args.only == "config1":
            out = _time_single(V, torch, "gauss_sym", W.gauss_sym_params(0.1), 4, 50, 100_000, "fp64",
                               args.steps, warm=args.warmup)
        elif args.only == "fp64":
            out = {fam: _time_single(V, torch, fam, p, D, NBINS, NEVENTS, "fp64", args.steps, warm=args.warmup)
                   for fam, p in _integrals()}
        elif args.only == "strat":
            out = {fam: _time_strat(V, torch, fam, p, D, NBINS, NEVENTS, PRECISION)
                   for fam, p in _integrals()}
        elif args.only == "lo_pdf":
            out = _time_lo_pdf(V, torch)
        elif args.only == "user":
            out = _time_user(V, torch)
        elif args.only == "lo":
            out = _time_single(V, torch, "lo", W.lo_params(), 3, 100, 100_000_000, "fp32_kahan",
                               args.steps, warm=args.warmup)
        else:
            out = {("rate_%d" % int(r)): _serving(V, rate=r, n_requests=serving_requests(r), target=1e-4,
                                                  budget=10 ** 9) for r in SERVING_RATES}
            out["poisson_batched_vs_fp64"] = _serving_compare(V, rate=100.0, n_requests=100, target=1e-4,
                                                              budget=10 ** 9)
        print(json.dumps({"only": args.only, **out}))
        return 0
    if world > 1:
        dist.init_process_group("nccl")
    from paper_2010_09341_gb300 import build as B
    if rank == 0:
        B.build()
    if world > 1:
        dist.barrier()
    from paper_2010_09341_gb300 import vegas as V

    stream = torch.cuda.current_stream()
    ctxs = []
    for k, (fam, p) in enumerate(_integrals()):
        cfg = V.Config(n_dim=D, n_events=NEVENTS, n_bins=NBINS, alpha=ALPHA, seed=0,
                       integral_id=rank * 2 + k, precision=PRECISION)
        ctxs.append(V.vegas_create(cfg, fam, p, stream=stream))
    samples_per_step = NEVENTS * len(ctxs)
    l2_flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def step():
        # both integrals: each one's sampling launch, then one launch for both
        # iteration results and refinements
        V.vegas_step_many(ctxs)

    def profile(on):
        for c in ctxs:
            V.vegas_profile(c, on)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    time.sleep(0.3)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    for k in range(args.steps):
        l2_flush.zero_()  # L2 flush between steps, outside the step events
        # CUDA events around the sampling launches of every PROFILE_EVERY-th
        # step give the kernel durations (an event pair between two launches
        # costs the step about 2 us)
        prof = k % PROFILE_EVERY == 0
        if prof:
            profile(True)
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
        if prof:
            profile(False)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = sum(step_ms)
    kern_ms = {c.family: V.vegas_profile_read(c) for c in ctxs}
    t = torch.tensor([total_ms], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    max_ms = float(t.item())
    value = world * samples_per_step * args.steps / (max_ms / 1e3)

    # ---- roofline of the dominant kernel (the sampling kernel)
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    sms = props.multi_processor_count
    clk_max_hz = (clk.get("sm_max_mhz") or 2070.0) * 1e6
    per_fam = {}
    ach_ops = 0.0      # algorithmic ops executed by the timed sampling launches
    roof_s = 0.0       # time those launches would take at the roofline
    kern_total_ms = 0.0
    for c in ctxs:
        ms = kern_ms[c.family]
        mean_ms = sum(ms) / max(1, len(ms))
        ops = ops_per_sample(c.family, D, PRECISION)
        bounds = roofline_samples_per_s(ops, sms, clk_max_hz)
        roof = min(bounds.values())
        ach = NEVENTS / (mean_ms / 1e3)
        per_fam[c.family] = {"kernel_ms": mean_ms, "samples_per_s": ach, "ops_per_sample": ops,
                             "roofline_samples_per_s": roof,
                             "bound_pipe": min(bounds, key=bounds.get),
                             "frac": ach / roof}
        ach_ops += ops["total"] * NEVENTS * len(ms)
        roof_s += NEVENTS * len(ms) / roof
        kern_total_ms += sum(ms)
    achieved_gops = ach_ops / (kern_total_ms / 1e3) / 1e9
    peak_gops = ach_ops / roof_s / 1e9
    roofline = {"bound": "alu", "achieved": achieved_gops, "peak": peak_gops, "unit": "Gop/s",
                "frac": achieved_gops / peak_gops, "traffic": _traffic_from_profile(),
                "kernel": "vegas_sample_kernel", "peak_basis":
                "min over pipes: issue 128 slots/clk/SM with a 32x32->64 multiply costing 4 slots, FP64 %.2f TFLOP/s, MUFU 32/clk/SM; %d SMs x %.0f MHz (max clock)"
                % (FP64_TFLOPS_NOMINAL, sms, clk_max_hz / 1e6), "per_integral": per_fam}

    # ---- end to end through the public API with host buffers
    # Every step of every integral ships its grid from pinned host memory to
    # the device (vegas_set_grid), runs vegas_step, and reads the combined
    # result and the refined grid back into pinned memory (vegas_result,
    # vegas_get_grid); the next step ships that grid back.  The two integrals
    # live on two streams and are pipelined: while one's step runs on the GPU,
    # the host reads the other's result and grid and enqueues its next step,
    # so the GPU always has work queued.
    e2e = None
    if args.e2e_steps > 0:
        streams = [torch.cuda.Stream() for _ in ctxs]
        ectx, grids = [], []
        for k, ((fam, p), s) in enumerate(zip(_integrals(), streams)):
            cfg = V.Config(n_dim=D, n_events=NEVENTS, n_bins=NBINS, alpha=ALPHA, seed=0,
                           integral_id=rank * 2 + k, precision=PRECISION)
            c = V.vegas_create(cfg, fam, p, stream=s)
            g = torch.empty((D, NBINS + 1), dtype=torch.float64, pin_memory=True).numpy()
            V.vegas_get_grid(c, out=g)
            ectx.append(c)
            grids.append(g)

        def e2e_run(steps):
            for c, g in zip(ectx, grids):
                V.vegas_set_grid(c, g)         # host -> device: grid state
                V.vegas_step(c, sync=False)    # sample, finalize + refine
            res = None
            for k in range(steps):
                res = []
                for c, g in zip(ectx, grids):
                    res.append(V.vegas_result(c))  # device -> host: combined result (waits for c)
                    V.vegas_get_grid(c, out=g)     # device -> host: refined grid
                    if k + 1 < steps:              # c's next step, while the other integral runs
                        V.vegas_set_grid(c, g)
                        V.vegas_step(c, sync=False)
            return res

        e2e_run(3)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        e2e_run(args.e2e_steps)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        tt = torch.tensor([dt], dtype=torch.float64, device="cuda")
        if world > 1:
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        dt = float(tt.item())
        gbytes = sum(g.nbytes for g in grids)
        rbytes = len(ectx) * ctypes_sizeof_result()
        e2e = {"value": world * samples_per_step * args.e2e_steps / dt, "unit": UNIT,
               "h2d_bytes_per_step": gbytes, "d2h_bytes_per_step": gbytes + rbytes,
               "steps": args.e2e_steps,
               "path": "per integral and step, each integral on its own stream: vegas_set_grid(pinned host "
                       "grid) + vegas_step, then vegas_result (to host) + vegas_get_grid(into pinned host grid); "
                       "the two integrals pipelined (one's host round trip while the other's step runs)"}

    # ---- the other workloads (rank 0 only)
    extra = None
    if rank == 0 and not args.no_extra:
        from paper_2010_09341_gb300 import workloads as W
        extra = {}
        extra["config1_fp64_d4_gauss"] = _time_single(
            V, torch, "gauss_sym", W.gauss_sym_params(0.1), 4, 50, 100_000, "fp64", 5)
        for fam, p in _integrals():
            extra["config2_fp64_path_" + fam] = _time_single(V, torch, fam, p, D, NBINS, NEVENTS,
                                                             "fp64", 3)
            extra["config2_fp32_kahan_" + fam] = _time_single(V, torch, fam, p, D, NBINS, NEVENTS,
                                                              "fp32_kahan", 10)
        for fam, p in _integrals():
            extra["stratified_hybrid_" + fam] = _time_strat(V, torch, fam, p, D, NBINS, NEVENTS,
                                                            PRECISION)
        extra["user_integrand_genz_gauss_d8"] = _time_user(V, torch)
        extra["config3_lo_fp32_kahan"] = _time_single(V, torch, "lo", W.lo_params(), 3, 100,
                                                      100_000_000, "fp32_kahan", 10)
        extra["config3_lo_pdf_grid_fp32_kahan"] = _time_lo_pdf(V, torch)
        extra["config4_batched"] = _time_batched(V, torch)
        for rate in SERVING_RATES:
            extra["config5_serving_rate_%d" % int(rate)] = _serving(
                V, rate=rate, n_requests=serving_requests(rate), target=1e-4, budget=10 ** 9)
        extra["config5_poisson_batched_vs_fp64"] = _serving_compare(V, rate=100.0, n_requests=100,
                                                                    target=1e-4, budget=10 ** 9)

    # ---- CPU baseline: the oracle on this host's cores (rank 0, N = 1)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        threads = os.cpu_count() or 1
        rate, n, dt = oracle_samples_per_s(args.cpu_seconds, threads)
        rate1, n1, dt1 = oracle_samples_per_s(min(3.0, args.cpu_seconds), 1)
        cpu = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": "%d samples (half per integral), iteration 0 on the uniform grid, %.1f s"
               % (n, dt),
               "single_thread": {"value": rate1, "unit": UNIT, "cores": 1,
                                 "sample": "%d samples (half per integral), iteration 0 on the "
                                           "uniform grid, %.1f s" % (n1, dt1)}}

    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": max_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 (FP64 accumulators)",
            "data": "synthetic",
            "config": dict(CONFIG, **{
                "l2": "flushed between steps (256 MiB write outside the step events); the kernel reads no HBM inputs",
                "parallelism": "replicas" if world > 1 else "single GPU"}),
            "method": {"precision": PRECISION, "samples_per_step": samples_per_step,
                       "step": "one iteration of both integrals (vegas_step_many): each one's sampling launch, then one finalize + refine launch for both",
                       "kernel_timing": "CUDA events around the sampling launches of every %dth timed step" % PROFILE_EVERY},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "extra": extra,
            "gpu_launches": args.steps * (len(ctxs) + 1),
            "clocks": clk,
        }
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
