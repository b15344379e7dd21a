#!/usr/bin/env python3
"""Benchmark: u ubar -> n gamma |M|^2 phase-space points/s on GB300.

Default workload (one step = one pass of the whole hot path over one batch):
u ubar -> 4 gamma, 1,048,576 points per GPU per step, sqrt(s-hat) from the toy
PDF x^(-1/2)(1-x)^3 at 14 TeV with sqrt(s-hat) > 100 GeV, cuts pT > 20 GeV,
|eta| < 2.5, Delta R > 0.4, all 64 helicities, FP32 spinor chain with FP64
RAMBO and double-double accumulation -- RNG, sampling, RAMBO, cuts, |M|^2,
weights and the Monte Carlo sums all run in one fused kernel (heget_xsec).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl heget|reference]

Multi-GPU (torchrun): rank r takes the contiguous point range
[r N, (r+1) N) of every step (weak scaling, no data-path collective; the
barrier and max-over-ranks timing use torch.distributed).
--impl reference times the FP64 CPU oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_PHOTONS = 4
POINTS = 1 << 20
SEED = 0x0908440300000002
METRIC = ("u ubar -> n gamma |M|^2 phase-space points/s (points whose |M|^2 is evaluated, i.e. that pass the cuts; "
          "n=4 workload; FP32 chain, FP64 phase space + accumulation)")
WORKLOAD = ("u ubar -> 4 gamma, 1,048,576 points/step/GPU, toy-PDF sqrt(s-hat) = 14 TeV sqrt(x1 x2) > 100 GeV "
            "with x ~ x^-1/2 (1-x)^3, cuts pT>20 GeV |eta|<2.5 dR>0.4, all 64 helicities")
PATH = ("24 orderings on the prefix tree with the two-ended finish, FP32 chain + FP64 RAMBO/cuts/denominators "
        "+ double-double sigma accumulation")
PATH_ORACLE = "FP64 CPU oracle: each of the 24 orderings from scratch with 4x4 Dirac matrices, compensated sums"


# Peaks derived from unit counts and the maximum SM clock (GB300: 152 SMs at
# 2.07 GHz; per SM and clock 128 FP32 FMA lanes and 2 FP64 FMA lanes), in
# TFLOP/s (an FMA counts 2 flops).
SMS, SM_GHZ = 152, 2.07
FP32_PEAK = SMS * 128 * 2 * SM_GHZ / 1e3
FP64_PEAK = SMS * 2 * 2 * SM_GHZ / 1e3
# FP64 flops executed per point by the fused n = 4 FP32 step (DFMA x 2 +
# DADD + DMUL, thread-level predicated-on counts from ncu on 262,144 points
# of this workload): sqrt(s-hat), RAMBO, cuts, and for the points that pass
# the cuts the denominators, records, weights and double-double sums.
# FP64_INSTR_PER_POINT: the same as instructions (DFMA + DADD + DMUL), each
# taking one slot of the FP64 pipe, 2 per SM and clock.
FP64_FLOPS_PER_POINT = {4: 671}
FP64_INSTR_PER_POINT = {4: 516.4}
# DRAM bytes per launch of that kernel (ncu dram__bytes_read.sum +
# dram__bytes_write.sum): its inputs come from the counter-based generator,
# so this is code, constant tables and block partials, the same at any size.
FP64_STEP_TRAFFIC = {4: 152832}


def roofline(n, N, kern_s, peak32_meas, peak64_meas, n_eval=None, subset=False):
    """Roofline of the fused step's kernel.  At n <= 4 the FP64 pipe binds
    (the phase space is FP64 by design; one SM retires 2 DFMA per clock
    against 128 FFMA), above that the FP32 tree does.  n_eval: points whose
    amplitudes were evaluated (those that pass the cuts).  subset: the step
    ran the subset recursion (its own flop count, FP32 pipe)."""
    fpp = subset_flops_per_point(n) if subset else tree_flops_per_point(n)
    tree = fpp * (N if n_eval is None else n_eval) / kern_s / 1e12
    fp32 = {"pipe": "fp32 fma", "achieved": tree, "peak": FP32_PEAK, "frac": tree / FP32_PEAK,
            "flops_per_point": fpp, "measured_peak": peak32_meas,
            "frac_of_measured": tree / peak32_meas}
    if subset:
        return {"bound": "alu", **fp32, "unit": "TFLOP/s", "traffic": None,
                "kernel": f"xsec_ws_kernel<float,{n}> (subset recursion)",
                "peak_source": "152 SMs x 128 FP32 FMA/clk x 2 flops x 2.07 GHz"}
    kern = f"xsec_ws_kernel<float,{n}>" if n <= 5 else f"xsec_kernel<float,{n},{ {6: 160, 7: 224}.get(n, 256)}>"
    if n in FP64_FLOPS_PER_POINT:
        a64 = FP64_FLOPS_PER_POINT[n] * N / kern_s / 1e12
        return {"bound": "alu", "pipe": "fp64", "achieved": a64, "peak": FP64_PEAK, "unit": "TFLOP/s",
                "frac": a64 / FP64_PEAK, "traffic": FP64_STEP_TRAFFIC.get(n), "kernel": kern,
                "flops_per_point": FP64_FLOPS_PER_POINT[n],
                "peak_source": "152 SMs x 2 FP64 FMA/clk x 2 flops x 2.07 GHz",
                "measured_peak": peak64_meas, "frac_of_measured": a64 / peak64_meas,
                "fp64_issue_frac": FP64_INSTR_PER_POINT[n] * N / kern_s / (SMS * 2 * SM_GHZ * 1e9),
                "fp32_tree": fp32}
    return {"bound": "alu", **fp32, "unit": "TFLOP/s", "traffic": None, "kernel": kern,
            "peak_source": "152 SMs x 128 FP32 FMA/clk x 2 flops x 2.07 GHz"}


def subset_flops_per_point(n: int) -> int:
    """FP32 flops of the subset recursion per point, met in the middle at
    m = n // 2 (an FMA counts 2 flops; a current term r.E or E.c and a Q
    product are 12 FMA each, a closing J.R product 8): J currents of sizes
    1..m (sizes >= 2: k terms and the Q product; size 1: the Q product), K
    currents of sizes 1..n-m-1 (the same), R currents of size n-m (n-m terms,
    no Q; at n = 2 none), and the contraction over the C(n, m) sets T for all
    2^n helicity configurations."""
    m, mk = n // 2, n - n // 2
    fma = 0
    for k in range(1, m + 1):
        fma += math.comb(n, k) * (1 << k) * (12 * k + 12 if k >= 2 else 12)
    for k in range(1, mk):
        fma += math.comb(n, k) * (1 << k) * (12 * k + 12 if k >= 2 else 12)
    if mk >= 2:
        fma += math.comb(n, mk) * (1 << mk) * 12 * mk
    fma += math.comb(n, m) * (1 << n) * 8
    return 2 * fma


def helas4_flops_per_point(n: int) -> int:
    """For comparison only: the same per-helicity prefix tree in the paper's
    4-component form, for each of the 2^(n+1) helicities with s2 = -s1 (the
    others vanish exactly).  A step applies the vertex eps-slash and the
    propagator q-slash to a 4-spinor -- in the chiral basis each is two 2x2
    complex products, 8 complex multiplies and 4 adds = 56 flops -- then the
    couplings and 1/q^2 (8 flops each): 128 flops.  A closure vbar eps-slash
    psi is 56 + a 4-term complex dot product (30) + the coupling (2) = 88.
    Steps per helicity: sum_{l=1}^{n-1} n!/(n-l)!; closures: n!."""
    f = math.factorial(n)
    steps = sum(f // math.factorial(n - l) for l in range(1, n))
    return (1 << (n + 1)) * (128 * steps + 88 * f)


def tree_flops_per_point(n: int, fp64: bool = False) -> int:
    """Flops of the ordering tree per point: 2^n helicity lanes, each doing
    sum_{l=2}^{n-1} n!/(n-l)! chain steps (28 flops: r . M, 2x2 complex) and n!
    closures (16 flops).  From n = 4 the walk stops two photons short and
    closes against per-point pair columns: the steps of level n - 1 go, and
    n(n-1) 4 pair columns (two 2-vector products, 32 flops) are formed."""
    f = math.factorial(n)
    two_ended = n >= 4
    last = n - 1 if two_ended else n
    steps = sum(f // math.factorial(n - l) for l in range(2, last))
    pairs = n * (n - 1) * 4 * 32 if two_ended else 0
    return (1 << n) * (28 * steps + 16 * f) + pairs


def dist_info():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled every 200 ms in the background."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self):
        self.proc = None
        # raw samples: HEGET_CLOCKS_CSV if set (to keep them), else a temporary file
        self.path = os.environ.get("HEGET_CLOCKS_CSV") or os.path.join(tempfile.gettempdir(),
                                                                         f"heget_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            if os.path.dirname(self.path):
                os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader",
                                          "-lms", "200"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except OSError:   # no nvidia-smi: no clock record
            self.proc = None
            if getattr(self, "fh", None):
                self.fh.close()
                if not os.environ.get("HEGET_CLOCKS_CSV"):
                    os.remove(self.path)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        with open(self.path) as fh:
            lines = fh.readlines()
        if not os.environ.get("HEGET_CLOCKS_CSV"):
            os.remove(self.path)
        return self.summarise(lines)

    @staticmethod
    def summarise(lines):
        """Median SM clock, the largest max clock and the throttle reasons
        seen Active, from nvidia-smi CSV lines in FIELDS order (None if no
        line parses)."""
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1].split()[0]))
                mx.append(float(f[2].split()[0]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_baseline(n, seconds=12.0, sampler=None, cut=None, seed=SEED, N_cap=None, single=True, exact=None):
    """The FP64 oracle, as it stands, on the host cores: a bounded sample of
    the same workload (consecutive point indices of the same seed), about
    `seconds` of work, or exactly `exact` points.  Its value counts the
    points whose |M|^2 is evaluated (those that pass the cuts; the oracle
    skips the others as the device does).  Returns the baseline record and the
    sample's weights (for the error columns)."""
    import oracle as O
    O.build()
    threads = os.cpu_count() or 1
    S = sampler if sampler is not None else O.toy_pdf()
    Cc = cut if cut is not None else O.cuts()
    import numpy as np
    probe = exact if exact else (threads if n >= 7 else 256)
    t0 = time.perf_counter()
    w, mask, _ = O.event_weights(n, seed, 0, probe, S, Cc, threads=threads)
    dt = time.perf_counter() - t0
    N = probe
    if not exact and dt < 0.5 * seconds:   # extend the sample to about `seconds` of work
        more = max(probe, int(probe * (seconds - dt) / max(dt, 1e-3)))
        if N_cap:
            more = max(0, min(more, N_cap - probe))
        if more:
            t1 = time.perf_counter()
            w2, m2, _ = O.event_weights(n, seed, probe, more, S, Cc, threads=threads)
            dt += time.perf_counter() - t1
            w = np.concatenate([w, w2])
            mask = np.concatenate([mask, m2])
            N += more
    npass = int(mask.sum())
    rec = {"value": npass / dt, "unit": "points/s", "cores": threads, "kind": "oracle",
           "generated_points_per_s": N / dt,
           "sample": f"points 0..{N - 1} of the n={n} workload (seed {seed:#x}), {npass} pass the cuts and have "
                     f"|M|^2 evaluated, {threads} OpenMP threads, {dt:.1f} s"}
    # one core as well, on the first points of the same sample (about 2 s of work)
    n1 = min(N, int(N / dt / threads * 2.0))
    if single and n1 >= 4:
        t1 = time.perf_counter()
        _, m1, _ = O.event_weights(n, seed, 0, n1, S, Cc, threads=1)
        d1 = time.perf_counter() - t1
        rec["single_thread"] = {"value": int(m1.sum()) / d1, "unit": "points/s", "cores": 1,
                                "sample": f"points 0..{n1 - 1}, 1 thread, {d1:.1f} s"}
    return rec, w


def run_reference(args):
    ws, rank, _ = dist_info()
    if rank != 0:
        return
    import oracle as O
    O.build()
    threads = os.cpu_count() or 1
    S, Cc = O.toy_pdf(), O.cuts()
    per_step = args.ref_points
    for w in range(args.warmup):
        O.event_weights(N_PHOTONS, SEED, w * per_step, min(per_step, 64), S, Cc, threads=threads)
    t0 = time.perf_counter()
    evaluated = 0
    for k in range(args.steps):
        _, mask, _ = O.event_weights(N_PHOTONS, SEED + k, 0, per_step, S, Cc, threads=threads)
        evaluated += int(mask.sum())
    dt = time.perf_counter() - t0
    value = evaluated / dt   # points whose |M|^2 is evaluated (they pass the cuts), as the device arm counts
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "points/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (Philox counter RNG from a seed)",
            "config": {"workload": WORKLOAD.replace("1,048,576", f"{per_step} (bounded CPU sample)"),
                       "n": N_PHOTONS, "points_per_step": per_step, "path": PATH_ORACLE},
            "events_per_s": per_step * args.steps / dt,
            "cpu_baseline": {"value": value, "unit": "points/s", "cores": threads, "kind": "oracle",
                             "sample": f"{per_step} points per step of the n={N_PHOTONS} workload, "
                                       f"{evaluated} of them with |M|^2 evaluated over the {args.steps} steps"},
            "e2e": {"value": value, "unit": "points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def time_xsec(H, ctx, n, N, sampler, precision, steps, stream, seed=SEED, i0=0, flush=None, result=None,
              detail=False):
    """Device time per step (ms) of heget_xsec_launch + heget_xsec_finalize,
    CUDA events on the launching stream, L2 flushed between steps.  result:
    a list that receives the last step's heget_xsec_result.  detail: return
    (step ms, kernel ms, evaluated points per step) instead, the kernel time
    between the launch's events and the evaluated points from every step's
    own result."""
    import torch
    res = torch.zeros((max(1, steps), 80), dtype=torch.uint8, device="cuda")
    for w in range(2):
        H.heget_xsec_launch(ctx, n, seed + 77 + w, i0, N, sampler, precision, stream=stream)
        H.heget_xsec_finalize(ctx, res[0], stream=stream)
    stream.synchronize()
    total = kern = 0.0
    for k in range(steps):
        if flush is not None:
            flush.add_(1)
            stream.wait_stream(torch.cuda.current_stream())
        a, b, c = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        a.record(stream)
        H.heget_xsec_launch(ctx, n, seed + k, i0, N, sampler, precision, stream=stream)
        b.record(stream)
        H.heget_xsec_finalize(ctx, res[k], stream=stream)
        c.record(stream)
        c.synchronize()
        total += a.elapsed_time(c)
        kern += a.elapsed_time(b)
    rs = [H.result_from_tensor(res[k]) for k in range(steps)]
    if result is not None:
        result.append(rs[-1])
    if detail:
        return total / steps, kern / steps, sum(r.n_pass for r in rs) / steps
    return total / steps


def time_amp2_subset(H, ctx, n, M, sampler, stream, flush, steps=5):
    """Points/s of heget_amp2 (FP32, the context's algorithm) on M phase-space
    points of the sampler, device time by CUDA events with L2 flushed between
    steps; the momenta are generated beforehand, outside the timed region."""
    import torch
    mom = torch.empty(M * (n + 2) * 4, dtype=torch.float64, device="cuda")
    H.heget_phase_space_ex(ctx, SEED + 321, 0, M, n, sampler, momenta=mom, stream=stream)
    amp = torch.empty(M, dtype=torch.float64, device="cuda")
    for _ in range(3):
        H.heget_amp2(ctx, n, M, mom, amp, precision=H.HEGET_FP32, stream=stream)
    stream.synchronize()
    ts = []
    for _ in range(steps):
        flush.add_(1)
        stream.wait_stream(torch.cuda.current_stream())
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        H.heget_amp2(ctx, n, M, mom, amp, precision=H.HEGET_FP32, stream=stream)
        b.record(stream)
        b.synchronize()
        ts.append(a.elapsed_time(b))
    return M / (sorted(ts)[len(ts) // 2] * 1e-3)


HIST_SPECS = [(0, 50, 20.0, 520.0), (1, 50, 20.0, 520.0), (2, 50, -2.5, 2.5), (3, 40, 0.4, 8.4),
              (4, 40, 0.4, 8.4)]


def time_hist(H, ctx, n, N, sampler, stream, seed, i0=0, flush=None, steps=5):
    """Device time (CUDA events) of heget_hist over the N events of one step,
    with that step's FP32 weights, L2 flushed between steps; points/s."""
    import torch
    res = torch.zeros(80, dtype=torch.uint8, device="cuda")
    w = torch.empty(N, dtype=torch.float64, device="cuda")
    out = torch.empty(H.hist_bins(HIST_SPECS), dtype=torch.float64, device="cuda")
    H.heget_xsec_async(ctx, n, seed, i0, N, sampler, H.HEGET_FP32, res, w, stream=stream)
    H.heget_hist(ctx, n, seed, i0, N, sampler, w, HIST_SPECS, out, stream=stream)
    stream.synchronize()
    total = 0.0
    for _ in range(steps):
        if flush is not None:
            flush.add_(1)
            stream.wait_stream(torch.cuda.current_stream())
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        H.heget_hist(ctx, n, seed, i0, N, sampler, w, HIST_SPECS, out, stream=stream)
        b.record(stream)
        b.synchronize()
        total += a.elapsed_time(b)
    ms = total / steps
    return {"points_per_s": N / (ms * 1e-3), "ms_per_step": ms, "steps": steps,
            "histograms": "max pT, pT, eta (50 bins each), Delta R of every pair, smallest Delta R (40 bins each)",
            "note": "heget_hist on the events of one step with its FP32 weights: momenta regenerated on the "
                    "device, double-double bin sums in a fixed order (Sec. 5, Fig. 2)"}


# ---------------------------------------------------------------------------
# serving: a Poisson trace of mixed requests through the request server
# ---------------------------------------------------------------------------

def serving_trace(R, rate, seed=0x5E4E, scaled=True):
    """R requests arriving as a Poisson process of `rate` per second: n uniform
    in 2..8, precision FP32 or FP64 with equal odds, toy-PDF sampler, and N
    log-uniform in [1e3, 1e6], divided by 8^(n-4) for n > 4 if `scaled` (the
    per-point cost grows ~10x per photon above n = 4).  Returns a list of
    dicts."""
    import numpy as np
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, R))
    n = rng.integers(2, 9, R)
    N = np.exp(rng.uniform(math.log(1e3), math.log(1e6), R))
    if scaled:
        N = N / 8.0 ** np.maximum(0, n - 4)
    N = np.maximum(1, N.astype(np.int64))
    prec = np.where(rng.random(R) < 0.5, 32, 64)
    return [dict(t=float(t[k]), n=int(n[k]), N=int(N[k]), precision=int(prec[k]), seed=SEED + 0x1000 + k)
            for k in range(R)]


def run_serving(H, ctx, trace, open_loop=True, timeout=300.0):
    """Submits the trace (at its arrival times, or all at once), waits for every
    result; latencies from the library's own submit/done stamps."""
    import threading
    S = H.sampler_toy_pdf()
    srv = H.heget_server_start(ctx)
    tickets = [None] * len(trace)
    try:
        def submitter():
            t0 = time.monotonic()
            for k, q in enumerate(trace):
                if open_loop:
                    dt = q["t"] - (time.monotonic() - t0)
                    if dt > 0:
                        time.sleep(dt)
                tickets[k] = H.heget_submit(srv, q["n"], q["seed"], q["N"], S, q["precision"])
        th = threading.Thread(target=submitter)
        th.start()
        th.join(timeout)
        results = [H.heget_wait(srv, t, timeout) for t in tickets]
    finally:
        H.heget_server_stop(srv)
    lat = sorted((r.t_done - r.t_submit) * 1e3 for r in results)
    span = max(r.t_done for r in results) - min(r.t_submit for r in results)
    pts = sum(q["N"] for q in trace)
    assert all(r.status == H.HEGET_OK for r in results)
    return {"p50_ms": lat[len(lat) // 2], "p99_ms": lat[min(len(lat) - 1, int(0.99 * len(lat)))],
            "max_ms": lat[-1], "points_per_s": pts / span, "span_s": span}


def run_sequential(H, ctx, trace, precision=None):
    """The same requests one after another, each a synchronous heget_xsec call
    (the plain per-request launch) at `precision` (None: the request's own)."""
    S = H.sampler_toy_pdf()
    t0 = time.perf_counter()
    for q in trace:
        H.heget_xsec(ctx, q["n"], q["N"], q["seed"], S, precision or q["precision"])
    dt = time.perf_counter() - t0
    return {"points_per_s": sum(q["N"] for q in trace) / dt, "span_s": dt}


def serving_section(H, ctx, R=400, rate=200.0, alg=0):
    H.heget_set_algorithm(ctx, alg)
    try:
        return _serving_section(H, ctx, R, rate)
    finally:
        H.heget_set_algorithm(ctx, H.HEGET_ALG_TREE)


def _serving_section(H, ctx, R, rate):
    trace = serving_trace(R, rate)
    warm = serving_trace(40, 2000.0, seed=0x3A11)
    run_serving(H, ctx, warm, open_loop=False)
    H.heget_xsec(ctx, 8, 16, 1, H.sampler_toy_pdf(), 64)
    closed = run_serving(H, ctx, trace, open_loop=False)
    open_ = run_serving(H, ctx, trace, open_loop=True)
    # the same requests arriving at 70 % of the saturated request rate
    cap = len(trace) / closed["span_s"]
    slow = [dict(q, t=q["t"] * rate / (0.7 * cap)) for q in trace]
    open_07 = run_serving(H, ctx, slow, open_loop=True)
    open_07["rate_per_s"] = 0.7 * cap
    seq64 = run_sequential(H, ctx, trace, precision=H.HEGET_FP64)
    seq_own = run_sequential(H, ctx, trace)
    return {"trace": f"{R} requests, Poisson {rate:g}/s, n uniform 2..8, FP32/FP64 1:1, toy PDF, "
                     "N log-uniform 1e3..1e6 / 8^(n-4) for n > 4",
            "points": sum(q["N"] for q in trace),
            "open_loop": open_, "saturated": closed, "open_loop_at_0.7_capacity": open_07,
            "sequential_fp64_plain": seq64, "sequential_own_precision": seq_own,
            "saturated_vs_sequential_fp64": closed["points_per_s"] / seq64["points_per_s"]}


def serving_cfg5(H, ctx, R=2000, rate=200.0):
    """The serving mix as specified: N log-uniform in 1e3..1e6 for every n (no
    scaling), R Poisson requests.  With the subset recursion: the saturated
    rate (every request submitted at once: the largest sustainable request
    rate), the open loop at 50 % of it, and sequential plain-FP64 calls.  The
    prefix tree cannot serve this trace in a bench run: its plain-FP64 n = 8
    requests alone take hours at its measured rate, which the line states
    from the per-n rates it measures here."""
    trace = serving_trace(R, rate, seed=0xCF65, scaled=False)
    S = H.sampler_toy_pdf()
    H.heget_set_algorithm(ctx, H.HEGET_ALG_SUBSET)
    try:
        run_serving(H, ctx, serving_trace(40, 2000.0, seed=0x3A12), open_loop=False)
        closed = run_serving(H, ctx, trace, open_loop=False, timeout=600.0)
        cap = len(trace) / closed["span_s"]
        half = [dict(q, t=q["t"] * rate / (0.5 * cap)) for q in trace]
        open_half = run_serving(H, ctx, half, open_loop=True, timeout=600.0)
        open_half["rate_per_s"] = 0.5 * cap
        seq64 = run_sequential(H, ctx, trace, precision=H.HEGET_FP64)
    finally:
        H.heget_set_algorithm(ctx, H.HEGET_ALG_TREE)
    # the tree's cost of the same trace from its rates on a probe per (n, precision)
    est = 0.0
    rates = {}
    for n in range(2, 9):
        for prec in (H.HEGET_FP32, H.HEGET_FP64):
            probe = {8: 256, 7: 2048}.get(n, 32768) if prec == H.HEGET_FP64 else {8: 4096, 7: 32768}.get(n, 262144)
            t0 = time.perf_counter()
            H.heget_xsec(ctx, n, probe, 0x5EED + n, S, prec)
            dt = time.perf_counter() - t0
            rates[f"n{n}_fp{prec}"] = probe / dt
            est += sum(q["N"] for q in trace if q["n"] == n and q["precision"] == prec) / (probe / dt)
    return {"trace": f"{R} requests, Poisson {rate:g}/s offered, n uniform 2..8, FP32/FP64 1:1, toy PDF, "
                     "N log-uniform 1e3..1e6 for every n",
            "points": sum(q["N"] for q in trace),
            "subset_recursion": {"saturated": closed, "max_sustainable_rate_per_s": cap,
                                 "open_loop_at_0.5_capacity": open_half,
                                 "sequential_fp64_plain": seq64,
                                 "saturated_vs_sequential_fp64": closed["points_per_s"] / seq64["points_per_s"]},
            "prefix_tree": {"served": False,
                            "gpu_seconds_estimate": est,
                            "note": "sequential GPU time of the trace with the paper's prefix tree, from its rates "
                                    "on a probe per (n, precision) (points/s in rates): beyond a bench run",
                            "rates": rates}}


# ---------------------------------------------------------------------------
# the four point workloads of the metric (u ubar -> n gamma, n = 2, 4, 6, 8)
# ---------------------------------------------------------------------------

CONFIGS = [
    # key, description, n, N, sampler (kind, args), cuts (pt, eta, dr), plain-FP64 timed points, FP32 timed
    # steps, error sample (points of the oracle's live sample, or the stored sample file)
    ("cfg1_n2", "u ubar -> 2 gamma, sqrt(s-hat) = 500 GeV fixed, 65,536 points, cuts pT>20 |eta|<2.5", 2, 65_536,
     ("fixed", 500.0), (20.0, 2.5, 0.0), 65_536, 5, 4096),
    ("cfg2_n4", "u ubar -> 4 gamma, toy-PDF sqrt(s-hat), 1,048,576 points, cuts pT>20 |eta|<2.5 dR>0.4", 4,
     1 << 20, ("toy",), (20.0, 2.5, 0.4), 1 << 20, 5, 4096),
    ("cfg3_n6", "u ubar -> 6 gamma, toy-PDF sqrt(s-hat), 1,048,576 points, same cuts", 6, 1 << 20, ("toy",),
     (20.0, 2.5, 0.4), 1 << 17, 3, 4096),
    ("cfg4_n8", "u ubar -> 8 gamma, sqrt(s-hat) uniform 200 GeV..2 TeV, 65,536 points, same cuts", 8, 65_536,
     ("uniform", 200.0, 2000.0), (20.0, 2.5, 0.4), 2048, 2, "tests/golden/oracle_weights_n8.txt"),
]


def read_stored_weights(path):
    """A stored oracle sample (tests/golden/gen_oracle_samples.py): its header
    fields and the weights of points 0 .. N-1."""
    import numpy as np
    head, w = [], []
    with open(os.path.join(ROOT, path)) as fh:
        for line in fh:
            if line.startswith("#"):
                head.append(line[1:].strip())
            elif line.strip():
                w.append(float(line.split()[3]))
    return head, np.array(w)


def _rel_errors(wg, w_or):
    import numpy as np
    nz = w_or != 0
    rel = np.abs(wg[nz] - w_or[nz]) / np.abs(w_or[nz])
    masks = bool(np.array_equal(wg != 0, nz))
    if not rel.size:
        return [0.0, 0.0], 0, masks
    return [float(np.median(rel)), float(rel.max())], int(nz.sum()), masks


def config_rows(H, ctx, stream, peak32, peak64, flush):
    """Per workload of the metric: FP32 (the paper's prefix tree) and plain
    FP64 points/s, the FP32 tree's fraction of the FP32 FMA peak from its own
    kernel time and flop count, the subset recursion beside them, and the
    FP32 and FP64 event weights' relative error against the FP64 oracle on a
    stated sample (outside the timed regions)."""
    import numpy as np
    import torch
    import oracle as O
    rows = {}
    for key, desc, n, N, smp, cut, n64, steps, err_sample in CONFIGS:
        S = {"fixed": lambda a: H.sampler_fixed(a[0]), "toy": lambda a: H.sampler_toy_pdf(),
             "uniform": lambda a: H.sampler_uniform(a[0], a[1])}[smp[0]](smp[1:])
        OS = {"fixed": lambda a: O.fixed(a[0]), "toy": lambda a: O.toy_pdf(),
              "uniform": lambda a: O.uniform(a[0], a[1])}[smp[0]](smp[1:])
        H.heget_set_params(ctx, pt_min=cut[0], eta_max=cut[1], dr_min=cut[2])
        tuned = None
        if key == "cfg3_n6":
            # the autotuner's choice of launch shape and tile for this workload (kept in the context)
            shape, tile, tms = H.heget_autotune_shape(ctx, n, H.HEGET_FP32, 1 << 18)
            threads, hrows, groups = H.heget_shape_info(n, H.HEGET_FP32, shape)
            tuned = {"shape": shape, "tile": tile, "probe_ms": tms, "probe_points": 1 << 18,
                     "shape_info": "the default launch shape" if shape == 0 else
                     f"tile kernel: {threads} threads, {hrows} helicity rows per lane, {groups} subtree groups"}
        ms32, k32, ev32 = time_xsec(H, ctx, n, N, S, H.HEGET_FP32, steps, stream, flush=flush, detail=True)
        if tuned:
            H.heget_set_shape(ctx, n, H.HEGET_FP32, 0)
            H.heget_set_tile(ctx, n, H.HEGET_FP32, 1, 0)
        ms64, k64, ev64 = time_xsec(H, ctx, n, n64, S, H.HEGET_FP64, 2 if n < 8 else 1, stream, flush=flush,
                                    detail=True)
        H.heget_set_algorithm(ctx, H.HEGET_ALG_SUBSET)
        # the subset recursion's launch (warp-specialised or a tile kernel) as the autotuner picks it
        sub_tile, sub_probe_ms = H.heget_autotune(ctx, n, H.HEGET_FP32, 1, min(N, 1 << 18))
        mss, ks, evs = time_xsec(H, ctx, n, N, S, H.HEGET_FP32, 3, stream, flush=flush, detail=True)
        H.heget_set_tile(ctx, n, H.HEGET_FP32, 1, 0)
        mss64, ks64, evs64 = time_xsec(H, ctx, n, N, S, H.HEGET_FP64, 2, stream, flush=flush, detail=True)
        amp_pps = time_amp2_subset(H, ctx, n, min(N, 1 << 18), S, stream, flush)
        H.heget_set_algorithm(ctx, H.HEGET_ALG_TREE)
        # relative errors of the event weights against the oracle
        if isinstance(err_sample, str):
            head, w_or = read_stored_weights(err_sample)
            oracle_rec = {"kind": "oracle", "sample": f"stored sample {err_sample} (points 0..{len(w_or) - 1}; "
                                                       + "; ".join(head[1:3]) + ")"}
        else:
            oracle_rec, w_or = cpu_baseline(n, sampler=OS, cut=O.cuts(*cut), single=False, exact=err_sample)
        M = len(w_or)
        errs = {}
        for prec in (H.HEGET_FP32, H.HEGET_FP64):
            w = torch.zeros(M, dtype=torch.float64, device="cuda")
            r = torch.zeros(80, dtype=torch.uint8, device="cuda")
            H.heget_xsec_async(ctx, n, SEED, 0, M, S, prec, r, w_out=w, stream=stream)
            stream.synchronize()
            errs[prec] = _rel_errors(w.cpu().numpy(), w_or)
        tf, sf = tree_flops_per_point(n), subset_flops_per_point(n)
        rows[key] = {
            "workload": desc, "n": n, "points": N, "pass_fraction": ev32 / N,
            "fp32": {"points_per_s": N / (ms32 * 1e-3), "evaluated_per_s": ev32 / (ms32 * 1e-3),
                     "ms_per_step": ms32, "kernel_ms": k32, "steps": steps, "autotuned": tuned,
                     "flops_per_evaluated_point": tf,
                     "frac_of_fp32_peak": tf * ev32 / (k32 * 1e-3) / (FP32_PEAK * 1e12),
                     "frac_of_measured_fp32_peak": tf * ev32 / (k32 * 1e-3) / (peak32 * 1e12),
                     "path": "prefix tree (the paper's ordering sum), FP32 chain"},
            "fp64_plain": {"points_per_s": n64 / (ms64 * 1e-3), "evaluated_per_s": ev64 / (ms64 * 1e-3),
                           "timed_points": n64, "kernel_ms": k64,
                           "frac_of_fp64_peak": tf * ev64 / (k64 * 1e-3) / (FP64_PEAK * 1e12)},
            "subset_recursion": {"fp32_points_per_s": N / (mss * 1e-3), "fp32_evaluated_per_s": evs / (mss * 1e-3),
                                 "fp64_points_per_s": N / (mss64 * 1e-3),
                                 "flops_per_evaluated_point": sf,
                                 "launch": "warp-specialised kernel" if sub_tile == 0 else f"tile kernel, {sub_tile}-point tiles",
                                 "autotune_probe_ms": sub_probe_ms,
                                 "fp32_frac_of_fp32_peak": sf * evs / (ks * 1e-3) / (FP32_PEAK * 1e12),
                                 "fp32_frac_of_measured_fp32_peak": sf * evs / (ks * 1e-3) / (peak32 * 1e12),
                                 "fp64_frac_of_fp64_peak": sf * evs64 / (ks64 * 1e-3) / (FP64_PEAK * 1e12),
                                 "amplitudes_only": {
                                     "points_per_s": amp_pps,
                                     "frac_of_fp32_peak": sf * amp_pps / (FP32_PEAK * 1e12),
                                     "frac_of_measured_fp32_peak": sf * amp_pps / (peak32 * 1e12),
                                     "path": "heget_amp2 FP32 on this workload's FP64 phase-space points (every "
                                             "point evaluated; input rows from HBM, FP64 invariants, FP32 recursion)"}},
            "rel_err_vs_oracle": {"fp32_median_max": errs[H.HEGET_FP32][0], "fp64_median_max": errs[H.HEGET_FP64][0],
                                  "points_compared": errs[H.HEGET_FP32][1],
                                  "masks_agree": errs[H.HEGET_FP32][2] and errs[H.HEGET_FP64][2],
                                  "sample": f"event weights of points 0..{M - 1} (seed {SEED:#x}) with |M|^2 "
                                            "evaluated, FP32 and FP64 tree against the FP64 oracle"},
            "oracle": oracle_rec,
        }
    H.heget_set_params(ctx)
    return rows


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="heget", choices=["heget", "reference"])
    ap.add_argument("--ref-points", type=int, default=2048)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-serving-cfg5", action="store_true",
                    help="leave out the serving mix as specified (2,000 unscaled requests; about a minute)")
    ap.add_argument("--e2e-steps", type=int, default=40)
    ap.add_argument("--n", type=int, default=N_PHOTONS, help="photons (profiling of smaller cases)")
    ap.add_argument("--points", type=int, default=POINTS, help="points per step per GPU")
    ap.add_argument("--alg", default="tree", choices=["tree", "subset"],
                    help="ordering-sum algorithm of the timed step (profiling of the subset recursion)")
    ap.add_argument("--sampler", default="toy", choices=["toy", "uniform"],
                    help="sqrt(s-hat) sampler of the timed step: toy PDF, or uniform 200 GeV..2 TeV")
    ap.add_argument("--no-configs", action="store_true",
                    help="leave out the per-workload rows (n = 2, 4, 6, 8; profiling runs)")
    ap.add_argument("--matrix", action="store_true", help=argparse.SUPPRESS)   # the rows are in the default line
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)

    import torch
    from paper_0908_4403_gb300 import build as B
    from paper_0908_4403_gb300 import heget as H

    ws, rank, local = dist_info()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    B.build()
    ctx = H.heget_create(local)
    stream = torch.cuda.Stream()
    from paper_0908_4403_gb300 import dist as D
    n, N = args.n, args.points
    i0, _ = D.shard(N * ws, ws, rank)   # weak scaling: N points per rank, contiguous ranges
    sampler = H.sampler_toy_pdf() if args.sampler == "toy" else H.sampler_uniform(200.0, 2000.0)
    if args.alg == "subset":
        H.heget_set_algorithm(ctx, H.HEGET_ALG_SUBSET)
    res = torch.zeros(80, dtype=torch.uint8, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")   # > 129 MB L2
    flush.random_(0, 255)

    peak32 = H.heget_measure_fma_peak(ctx, H.HEGET_FP32)
    peak64 = H.heget_measure_fma_peak(ctx, H.HEGET_FP64)

    with torch.cuda.stream(stream):
        for w in range(args.warmup):
            H.heget_xsec_launch(ctx, n, SEED + 1000 + w, i0, N, sampler, H.HEGET_FP32, stream=stream)
            H.heget_xsec_finalize(ctx, res, stream=stream)
    stream.synchronize()

    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
            torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler()
    clocks.start()
    time.sleep(0.3)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    res_steps = torch.zeros((args.steps, 80), dtype=torch.uint8, device="cuda")   # each step's own result
    for k in range(args.steps):
        flush.add_(1)   # evict L2 between timed steps (untimed)
        stream.wait_stream(torch.cuda.current_stream())
        a, b, c = evs[k]
        a.record(stream)
        H.heget_xsec_launch(ctx, n, SEED + k, i0, N, sampler, H.HEGET_FP32, stream=stream)
        b.record(stream)
        H.heget_xsec_finalize(ctx, res_steps[k], stream=stream)
        c.record(stream)
        torch.cuda.current_stream().wait_stream(stream)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    clock_info = clocks.stop()
    step_ms = sum(a.elapsed_time(c) for a, _, c in evs)
    kern_ms = sum(a.elapsed_time(b) for a, b, _ in evs)
    step_res = [H.result_from_tensor(res_steps[k]) for k in range(args.steps)]
    evaluated = float(sum(x.n_pass for x in step_res))   # points whose |M|^2 was evaluated, this rank
    if ws > 1:
        t = torch.tensor([step_ms, kern_ms], dtype=torch.float64, device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        step_ms, kern_ms = t.tolist()
        t = torch.tensor([evaluated], dtype=torch.float64, device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.SUM)
        evaluated = t.item()
    r = step_res[-1]
    if ws > 1:   # the job's cross section of the last step: per-rank sums combined in rank order
        r = D.allreduce_result(r, sampler.kind)

    H.heget_set_algorithm(ctx, H.HEGET_ALG_TREE)
    # the plain FP64 GPU kernel on the same workload (the comparison the
    # workload is quoted with)
    fp64_steps = max(3, min(20, args.steps // 20))
    ms64 = time_xsec(H, ctx, n, N, sampler, H.HEGET_FP64, fp64_steps, stream, seed=SEED + 5000, i0=i0,
                     flush=flush)

    # the same workload with the subset recursion (not the paper's method)
    H.heget_set_algorithm(ctx, H.HEGET_ALG_SUBSET)
    ms_sub = time_xsec(H, ctx, n, N, sampler, H.HEGET_FP32, max(5, min(50, args.steps // 8)), stream,
                       seed=SEED + 7000, i0=i0, flush=flush)
    ms_sub64 = time_xsec(H, ctx, n, N, sampler, H.HEGET_FP64, fp64_steps, stream, seed=SEED + 7500, i0=i0,
                         flush=flush)
    H.heget_set_algorithm(ctx, H.HEGET_ALG_TREE)

    # FP32 -> FP64 escalation at the accuracy target (off by default)
    H.heget_set_escalation(ctx, 1e-4)
    esc_res = []
    ms_esc = time_xsec(H, ctx, n, N, sampler, H.HEGET_FP32, max(5, min(50, args.steps // 8)), stream,
                       seed=SEED + 8000, i0=i0, flush=flush, result=esc_res)
    H.heget_set_escalation(ctx, 0.0)

    # kinematic distributions (Sec. 5, Fig. 2) of the same events: the step's
    # weights, then heget_hist regenerates the momenta and bins max pT, the
    # photons' pT and eta, every pair's Delta R and the smallest Delta R
    dist = time_hist(H, ctx, n, N, sampler, stream, seed=SEED + 8500, i0=i0, flush=flush)

    # end to end through the public API: heget_xsec per step (launch, fused
    # RNG -> sampler -> RAMBO -> cuts -> |M|^2 -> sums, result read back to a
    # host struct, synchronised); the step's inputs are its arguments
    e2e_seed = SEED + 9000 + (rank << 32)
    for w in range(3):
        H.heget_xsec(ctx, n, N, e2e_seed + w, sampler, H.HEGET_FP32)
    if ws > 1:
        torch.distributed.barrier()
    t0 = time.perf_counter()
    e2e_eval = 0
    for k in range(args.e2e_steps):
        e2e_eval += H.heget_xsec(ctx, n, N, e2e_seed + k, sampler, H.HEGET_FP32).n_pass
    e2e_s = time.perf_counter() - t0
    e2e_eval = float(e2e_eval)
    if ws > 1:
        t = torch.tensor([e2e_s], dtype=torch.float64, device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        e2e_s = t.item()
        t = torch.tensor([e2e_eval], dtype=torch.float64, device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.SUM)
        e2e_eval = t.item()

    serving = None
    if rank == 0 and ws == 1 and not args.no_serving:
        serving = serving_section(H, ctx)
        serving["subset_recursion"] = serving_section(H, ctx, alg=H.HEGET_ALG_SUBSET)
        if not args.no_serving_cfg5:
            serving["cfg5_as_specified"] = serving_cfg5(H, ctx)

    configs = None
    if rank == 0 and ws == 1 and not args.no_configs:
        configs = config_rows(H, ctx, stream, peak32, peak64, flush)

    if rank == 0:
        total_points = N * ws * args.steps
        value = evaluated / (step_ms * 1e-3)
        kern_s = kern_ms / args.steps * 1e-3
        line = {
            "metric": METRIC, "value": value, "unit": "points/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 chain + f64 phase space/accumulation",
            "data": "synthetic (on-device Philox4x32-10 counter RNG from a seed; toy PDF)",
            "config": {"workload": WORKLOAD if (n, N, args.sampler) == (N_PHOTONS, POINTS, "toy")
                       else f"n={n}, {N} points/step, {args.sampler} sqrt(s-hat)",
                       "n": n, "points_per_step": N * ws, "precision": "fp32",
                       "path": PATH if args.alg == "tree" else "subset recursion (HEGET_ALG_SUBSET), FP32",
                       "l2": "flushed between timed steps (256 MiB write, untimed)",
                       "compaction": "value counts the points whose |M|^2 is evaluated: those that pass the "
                                     "cuts (the others have weight 0 and no amplitude); events_per_s counts every "
                                     "generated point",
                       "parallelism": f"dp{ws} (point shards)"},
            "events_per_s": total_points / (step_ms * 1e-3),
            "pass_fraction": evaluated / total_points,
            "roofline": roofline(n, N, kern_s, peak32, peak64, n_eval=evaluated / ws / args.steps,
                                 subset=args.alg == "subset"),
            "gpu_launches": 2 * args.steps,
            "e2e": {"value": e2e_eval / e2e_s, "unit": "points/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 80, "events_per_s": N * ws * args.e2e_steps / e2e_s,
                    "path": "heget_xsec (synchronous public call): inputs (n, N, seed, sampler) travel as launch "
                            "arguments, the 80-byte result is copied to a host struct every step"},
            "fp64_plain": {"value": N / (ms64 * 1e-3), "unit": "points/s", "ms_per_step": ms64,
                           "steps": fp64_steps, "kernel": f"xsec_kernel<double,{n},256>"},
            "subset_recursion": {"fp32_points_per_s": N * ws / (ms_sub * 1e-3),
                                 "fp64_points_per_s": N * ws / (ms_sub64 * 1e-3),
                                 "note": "HEGET_ALG_SUBSET on the same workload: the ordering sum regrouped by "
                                         "photon set (not the paper's method; same |M|^2)"},
            "escalation": {"tau": 1e-4, "points_per_s": N * ws / (ms_esc * 1e-3),
                           "n_escalated_last_step": esc_res[0].n_escalated, "n_pass_last_step": esc_res[0].n_pass,
                           "note": "the same step with FP32 points whose error bound exceeds tau recomputed "
                                   "in FP64 (heget_set_escalation; off in the headline value)"},
            "distributions": dist,
            "kernel_ms_per_step": kern_ms / args.steps,
            "result_last_step": {"sigma_fb": r.sigma_fb, "err_fb": r.err_fb, "n_pass": r.n_pass,
                                 "accept": r.accept, "pass_fraction": r.n_pass / max(1, r.n_total)},
        }
        if clock_info:
            line["clocks"] = clock_info
        if serving:
            line["serving"] = serving
        if ws == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(n)[0]
        if configs:
            line["configs"] = configs
        print(json.dumps(line), flush=True)
    H.heget_destroy(ctx)
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
