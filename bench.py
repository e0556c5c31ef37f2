#!/usr/bin/env python
"""Benchmark of the batched Galactic-binary likelihood path on GB300.

One step = one 10,000-proposal posterior round on each of 16 frequency
windows (N = 128 / 256 bins, T = 2 yr, one injected binary per window at SNR
20-200, proposals from a Gaussian of 10x the Fisher width around it): the
mixed-precision log-likelihood of all 160,000 proposals (one persistent
launch), the 16 independence Metropolis-Hastings chains built from them, and
the certification that makes those chains the FP64 path's: the proposals whose
accept/reject decision the mixed error bound cannot settle are re-evaluated in
FP64 (gb_mh_certified).

Metric: GB logL evaluations per second (higher is better) of the certified
round (headline), of the same round without certification and of the plain
FP64 path, with |dlogL| of the mixed path against FP64 stated per SNR band, and
seconds per 10k-sample posterior round.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
  python bench.py --workload tiny|band|population|fullband   (the other
      configurations: one JSON line each with their own figures; not the
      headline line)

Under torchrun each rank runs its own replica of the workload (different
seed) on its own GPU with no collective on the data path (weak scaling); with
--shard the ranks share one workload's windows out instead (cost-balanced,
strong scaling).  Only the timing uses a barrier and a max over ranks.  Rank 0
prints one JSON line.
"""
import argparse
import json
import math
import os
import shutil
import subprocess
import sys
import threading
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2307_03763_gb300 import workloads as wk  # noqa: E402

METRIC = "GB logL evals/s (FP64 vs mixed, |dlogL| stated); s per 10k-sample posterior"
UNIT = "evals/s"
WORKLOAD = "posterior: 16 windows (N=128/256, f0 log-U[0.5,5] mHz), 10,000 proposals each, T=2 yr, dt=15 s"
L2_BYTES = 129 * 1024 * 1024
MAX_ITER = 2          # re-evaluation passes of the certified rounds


# ---------------------------------------------------------------------------
# workload construction (host; the template and its derivatives come from the
# library's own waveform kernel)
# ---------------------------------------------------------------------------

def build_inputs(ctx, seed, dev):
    wl = wk.posterior_windows(seed=seed)
    T = wl.T
    nwin = len(wl.windows)
    src = np.array([wl.sources[w][0] for w in range(nwin)])     # A = 1

    def templates(th):
        """gb_waveform (fp64) of rows th for every window's N, scattered on its bins."""
        outA = np.zeros((len(th), max(w[1] for w in wl.windows)), np.complex128)
        outE = np.zeros_like(outA)
        for w, (k0, W, N, doff, coff, nc) in enumerate(wl.windows):
            rows = [i for i in range(len(th)) if i % nwin == w]
            if not rows:
                continue
            hA, hE, q = ctx.waveform(torch.tensor(th[rows], device=dev), N, "fp64")
            hA, hE, q = hA.cpu().numpy(), hE.cpu().numpy(), q.cpu().numpy()
            for r, i in enumerate(rows):
                j = q[r] - N // 2 + np.arange(N) - k0
                ok = (j >= 0) & (j < W)
                outA[i, j[ok]] = hA[r, ok]
                outE[i, j[ok]] = hE[r, ok]
        return outA, outE

    def inner(aA, aE, bA, bE, w):
        k0, W, N, doff, _, _ = wl.windows[w]
        wa, we = wl.w_A[doff:doff + W], wl.w_E[doff:doff + W]
        return (4.0 / T) * (np.sum(wa * (aA[:W] * bA[:W].conj()).real) + np.sum(we * (aE[:W] * bE[:W].conj()).real))

    hA, hE = templates(src)
    for w in range(nwin):
        src[w, 4] = wl.meta["snr"][w] / math.sqrt(inner(hA[w], hE[w], hA[w], hE[w], w))
    # Fisher matrix F_ij = <d_i h|d_j h> by central differences of the templates
    scales = np.array([1 / T, 1 / T ** 2, 1, 1, 1, 1, 1, 1.0])
    sig = np.zeros((nwin, 8))
    J = []
    for i in range(8):
        step = 1e-4 * scales[i] * (src[:, 4] if i == 4 else 1.0)
        tp, tm = src.copy(), src.copy()
        tp[:, i] += step
        tm[:, i] -= step
        pA, pE = templates(tp)
        mA, mE = templates(tm)
        st = step if np.ndim(step) else np.full(nwin, step)
        J.append(((pA - mA) / (2 * st[:, None]), (pE - mE) / (2 * st[:, None])))
    for w in range(nwin):
        F = np.array([[inner(J[i][0][w], J[i][1][w], J[j][0][w], J[j][1][w], w) for j in range(8)]
                      for i in range(8)])
        # inverted in natural units (1/T, 1/T^2, rad, A): in SI units the entries
        # span ~70 decades, beyond a pseudo-inverse's relative cut-off
        sc = np.array([1 / T, 1 / T ** 2, 1, 1, src[w, 4], 1, 1, 1.0])
        sig[w] = np.sqrt(np.abs(np.diag(np.linalg.pinv(F * np.outer(sc, sc))))) * sc
    # data = noise + injected sources
    hA, hE = templates(src)
    dA, dE = wl.noise_A.copy(), wl.noise_E.copy()
    for w, (k0, W, N, doff, coff, nc) in enumerate(wl.windows):
        dA[doff:doff + W] += hA[w, :W]
        dE[doff:doff + W] += hE[w, :W]
    wl.meta["source"] = src.copy()
    wl.meta["fisher_sigma"] = sig.copy()
    rng = np.random.default_rng(wl.meta["proposal_seed"])
    theta = np.empty((wl.n_cand, 8))
    log_g = np.empty(wl.n_cand)
    for w, (k0, W, N, doff, coff, nc) in enumerate(wl.windows):
        theta[coff:coff + nc], log_g[coff:coff + nc] = wk.gaussian_proposals(src[w], 10 * sig[w], nc, rng)
    return wl, dA, dE, theta, log_g


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.rows = []

    def start(self):
        exe = shutil.which("nvidia-smi")
        if not exe:
            return
        self.proc = subprocess.Popen([exe, "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                      "--format=csv,noheader,nounits", "-lms", "100"],
                                     stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm = [float(r[0]) for r in self.rows if len(r) >= 8 and r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if len(r) >= 8 and r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows if len(r) >= 8 for k in range(4)
                          if r[4 + k].lower().startswith("active")})
        power = [float(r[2]) for r in self.rows if len(r) >= 8 and r[2].replace(".", "").isdigit()]
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(sm), "power_w_max": max(power) if power else None}


# ---------------------------------------------------------------------------
# algorithmic work of the likelihood kernel (counted from the algorithm)
# ---------------------------------------------------------------------------

def flops_per_eval(N, f_hz, T):
    """Floating-point operations of one evaluation (FMA = 2), mixed path.

    Per sample (counted from the algorithm as the kernel states it, a
    sincospi counted as 20): common double-word phase 108, three
    per-spacecraft phase factors 93, f and a 4, three arms with their two
    links 3 x (66 + 8 J), TDI, delay factor and the A/E projection 80; so
    483 + 24 J.  FFT 2 x 5 N log2 N; window inner products 26 per bin.
    J = 4 below 9.3 mHz (f/f* <= 0.489), 7 below 25.6 mHz.
    """
    xmax = f_hz / (299792458.0 / (2 * math.pi * 2.5e9))
    J = 4 if xmax <= 0.489 else 7 if xmax <= 1.34 else 10
    per_sample = 483 + 24 * J
    return N * per_sample + 2 * 5 * N * math.log2(N) + 26 * N


def flops_per_grad(N, f_hz, T):
    """Floating-point operations of one mixed-precision gradient (FMA = 2).

    The forward evaluation (as flops_per_eval, with 38 per window bin for the
    inner products and the weighted residual), the adjoint transform of both
    channels (2 x 5 N log2 N), and per sample the reverse-mode step: the
    sample's values again, with the transfer functions' X derivatives
    (508 + 48 J), and the adjoint arithmetic from the channel weights to the
    four parameter sums and the P, Q sums (555).
    """
    xmax = f_hz / (299792458.0 / (2 * math.pi * 2.5e9))
    J = 4 if xmax <= 0.489 else 7 if xmax <= 1.34 else 10
    forward = N * (483 + 24 * J) + 2 * 5 * N * math.log2(N) + 38 * N
    return forward + 2 * 5 * N * math.log2(N) + N * (508 + 48 * J + 555)


def source_sha256(sources):
    """SHA-256 of a kernel's code: the listed files (each up to its optional
    `until` marker) concatenated, without // comments and blank lines."""
    import hashlib
    region = ""
    for src in sources:
        text = open(os.path.join(ROOT, src["path"])).read()
        if src.get("until"):
            text = text.split(src["until"])[0]
        region += text
    region = "\n".join(ln.split("//")[0].rstrip() for ln in region.splitlines())
    region = "\n".join(ln for ln in region.splitlines() if ln.strip())
    return hashlib.sha256(region.encode()).hexdigest()


def profiled_traffic(name="loglik_mixed_posterior"):
    """DRAM bytes per launch of a kernel from its committed ncu counters
    (profiles/<name>.json: dram__bytes_read.sum + dram__bytes_write.sum of one
    captured launch), or None when the kernel's code changed since that
    capture (the hash of the source files the file lists differs)."""
    try:
        prof = json.load(open(os.path.join(ROOT, "profiles", name + ".json")))
        if prof.get("source_sha256") != source_sha256(prof["sources"]):
            return None
    except (OSError, ValueError, KeyError):
        return None
    return int(prof["traffic_bytes_per_launch"])


def flops_per_grad_fp64(N, f_hz, T):
    """Algorithmic floating-point operations of one FP64 gradient (FMA = 2), the
    same reverse-mode count as flops_per_grad with the FP64 path's per-sample
    forward work (flops_per_eval_fp64) and its link-series degrees J = 6, 8,
    12, 16: forward with 38 per window bin, the adjoint transform of both
    channels, and per sample 508 + 48 J + 555 for the reverse step.  The FP64
    kernel's reverse sweep recomputes the sample's forward values and
    evaluates the link transfer's derivative series beside it."""
    x = f_hz / (299792458.0 / (2 * math.pi * 2.5e9))
    J = 6 if x <= 0.22 else 8 if x <= 0.5 else 12 if x <= 1.3 else 16
    forward = N * (445 + 24 * J) + 2 * 5 * N * math.log2(N) + 38 * N
    return forward + 2 * 5 * N * math.log2(N) + N * (508 + 48 * J + 555)


def flops_per_eval_fp64(N, f_hz, T):
    """Floating-point operations of one evaluation of the FP64 path (FMA = 2,
    a sincos or sincospi counted as 20), counted from the algorithm as the
    FP64 kernel states it.  Per sample: three receiver phases (projection 6,
    phase in cycles 18, reduction and sincospi 22) 138; f and a 4; three arms
    (k.n 5, n.H.n 19, two links of 20 + 4 J each: argument, series in
    -4X^2, complex scaling and two complex products) 3 x (64 + 8 J); the delay
    factor by its short series and D^2, 27; X, Y, Z with (1 - D^2) 72; the A/E
    projection 12; so 445 + 24 J with J = 6, 8, 12, 16 by f/f* <= 0.22, 0.5,
    1.3, 2.35.  FFT 2 x 5 N log2 N; window inner products 32 per bin.
    """
    x = f_hz / (299792458.0 / (2 * math.pi * 2.5e9))
    J = 6 if x <= 0.22 else 8 if x <= 0.5 else 12 if x <= 1.3 else 16
    return N * (445 + 24 * J) + 2 * 5 * N * math.log2(N) + 32 * N


def fp64_peak_tflops(clock_mhz=2070.0):
    """FP64 peak from unit counts: 152 SMs x 2 FP64 FMA lanes x 2 flops x clock.
    Two lanes per SM (1/64 of the 128 FP32 lanes) is what GB300's nominal
    1.25 TFLOP/s dense FP64 implies at 2.07 GHz."""
    return 152 * 2 * 2 * clock_mhz * 1e6 / 1e12


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else platform)."""
    import platform
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.processor() or platform.machine()


# ---------------------------------------------------------------------------

def window_mix(wl):
    """One window of each template size N in the step, with the share of the
    step's evaluations that windows of that N hold."""
    total = sum(w[5] for w in wl.windows)
    mix = {}
    for w in wl.windows:
        if w[2] not in mix:
            mix[w[2]] = [w, 0]
        mix[w[2]][1] += w[5]
    return [(w, cnt / total) for w, cnt in mix.values()]


def cpu_rate(fn, wl, dA, dE, theta, seconds, n=1000):
    """Evaluations per second of fn (the oracle's loglik or its FFT variant)
    over the step's window mix: each distinct N timed on n proposals of one of
    its windows for about seconds / (number of N), combined by the step's
    shares (time per evaluation weighted by share)."""
    mix = window_mix(wl)
    t_per = 0.0
    for (k0, W, N, doff, coff, nc), share in mix:
        m = min(n, nc)
        win = [(k0, W, N, doff, 0, m)]
        th = theta[coff:coff + m]
        fn(win, dA, dE, wl.w_A, wl.w_E, th, wl.T)            # warm
        t0 = time.perf_counter()
        done = 0
        while True:
            fn(win, dA, dE, wl.w_A, wl.w_E, th, wl.T)
            done += m
            if time.perf_counter() - t0 > seconds / len(mix):
                break
        t_per += share * (time.perf_counter() - t0) / done
    return 1.0 / t_per, mix


def cpu_baseline(wl, dA, dE, theta, seconds=12.0):
    """The FP64 oracle as it stands (naive DFT), and the same with a radix-2
    FFT, timed on this host's cores on a bounded sample of the step's window mix."""
    from oracle import cpu_fft
    from oracle import gb as ogb
    rate, mix = cpu_rate(ogb.loglik, wl, dA, dE, theta, seconds)
    rate_fft, _ = cpu_rate(cpu_fft.loglik_fft, wl, dA, dE, theta, seconds)
    sample = ("1,000 proposals of one window of each N in the step (%s), each timed for ~%.0f s, "
              "weighted by the step's evaluations per N" %
              (", ".join("N=%d: %.0f%%" % (w[2], 100 * sh) for w, sh in mix), seconds / len(mix)))
    host = {"cores": torch.get_num_threads(), "cpu_count": os.cpu_count(), "cpu_model": cpu_model()}
    base = {"value": rate, "unit": UNIT, "kind": "oracle", "dft": "naive O(N^2)", "sample": sample, **host}
    fft = {"value": rate_fft, "unit": UNIT, "kind": "oracle steps with a radix-2 FFT (oracle/cpu_fft.py)",
           "dft": "radix-2 FFT", "sample": sample, **host}
    return base, fft


def run_reference(args, rank, world):
    """The oracle as it stands (CPU) on the same workload and metric: per step,
    1,000 proposals of one window of each N in the step (likelihood and chain),
    combined by the step's evaluations per N."""
    if rank != 0:
        return
    from oracle import gb as ogb
    from oracle import mh as omh
    wl = wk.posterior_windows()

    def on_window(s, w):
        k0, W, N, doff, _, _ = wl.windows[w]
        q, hA, hE = ogb.template(torch.tensor(s[None]), N, wl.T)
        j = int(q[0]) - N // 2 + np.arange(N) - k0
        ok = (j >= 0) & (j < W)
        a, e = np.zeros(W, np.complex128), np.zeros(W, np.complex128)
        a[j[ok]], e[j[ok]] = hA[0].numpy()[ok], hE[0].numpy()[ok]
        return a, e

    dA, dE = wl.noise_A.copy(), wl.noise_E.copy()
    srcs = []
    for w, (k0, W, N, doff, coff, nc) in enumerate(wl.windows):
        s = wl.sources[w][0].copy()
        a, e = on_window(s, w)
        hh = (4 / wl.T) * (np.sum(wl.w_A[doff:doff + W] * abs(a) ** 2) + np.sum(wl.w_E[doff:doff + W] * abs(e) ** 2))
        s[4] = wl.meta["snr"][w] / math.sqrt(hh)
        a, e = on_window(s, w)
        dA[doff:doff + W] += a
        dE[doff:doff + W] += e
        srcs.append(s)
    n = 1000
    rng = np.random.default_rng(1)
    parts = []
    for (k0, W, N, doff, coff, nc), share in window_mix(wl):
        w = [x[0] for x in wl.windows].index(k0)
        sig = np.array([0.3 / wl.T, 1e-19, 0.05, 0.05, 0.1 * srcs[w][4], 0.05, 0.05, 0.05])
        th, lg = wk.gaussian_proposals(srcs[w], sig, n, rng)
        parts.append(([(k0, W, N, doff, 0, n)], th, lg, wk.log_uniforms(n, rng), share))

    def part(p):
        win, th, lg, lu, _ = p
        l, _, _ = ogb.loglik(win, dA, dE, wl.w_A, wl.w_E, th, wl.T)
        omh.mh_independence(l.numpy(), lg, lu, 1.0)

    for _ in range(args.warmup):
        for p in parts:
            part(p)
    t_per = 0.0
    for p in parts:
        t0 = time.perf_counter()
        for _ in range(args.steps):
            part(p)
        t_per += p[4] * (time.perf_counter() - t0) / (args.steps * n)
    value = 1.0 / t_per
    sample = ("%d proposals of one window of each N in the step (%s) per step, likelihood and chain, "
              "weighted by the step's evaluations per N" %
              (n, ", ".join("N=%d: %.0f%%" % (p[0][0][2], 100 * p[4]) for p in parts)))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * n / value,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "kind": "oracle", "cores": torch.get_num_threads(),
                             "cpu_count": os.cpu_count(), "cpu_model": cpu_model(), "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# the other configurations (one GPU): their own figures, one JSON line each
# ---------------------------------------------------------------------------

def run_workload(args):
    """tiny: one N = 128 window, 1,000 candidates (FP64 and mixed logL);
    band: 512 windows over 0.3-20 mHz, N = 32..1024, 2k-20k candidates each,
    one persistent launch; population: 64 windows x 4,096 (N = 256), logL,
    adjoint gradient in both precisions, and 200 GA generations."""
    from paper_2307_03763_gb300 import api, build
    from paper_2307_03763_gb300.ga import GASearch
    build.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)

    def timed(fn, reps, warm=3, flush_l2=True):
        for _ in range(warm):
            fn()
        torch.cuda.synchronize(dev)
        ms = []
        for _ in range(reps):
            if flush_l2:
                flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            ms.append((a, b))
        torch.cuda.synchronize(dev)
        return float(np.mean([a.elapsed_time(b) for a, b in ms]))

    wl = {"tiny": wk.tiny_window, "band": wk.band_windows, "population": wk.population_windows}[args.workload]()
    ctx = api.Context(wl.T)
    T_ = lambda x, dt: torch.as_tensor(np.ascontiguousarray(x)).to(dev, dt)
    data = (T_(wl.noise_A, torch.complex128), T_(wl.noise_E, torch.complex128), T_(wl.w_A, torch.float64),
            T_(wl.w_E, torch.float64))
    theta = T_(wl.theta, torch.float64)
    n = wl.n_cand
    reps = max(3, min(args.steps, 20))
    clocks = ClockSampler(dev.index)
    clocks.start()
    tune = ctx.autotune(wl.windows, *data, theta, prec="mixed", reps=3)
    ms_mx = timed(lambda: ctx.loglik(wl.windows, *data, theta, prec="mixed"), reps)
    ms_64 = timed(lambda: ctx.loglik(wl.windows, *data, theta, prec="fp64"), 1 if n > 10 ** 6 else 3)
    l64 = ctx.loglik(wl.windows, *data, theta, prec="fp64")[0]
    lmx = ctx.loglik(wl.windows, *data, theta, prec="mixed")[0]
    dl = (lmx - l64).abs()
    line = {"metric": METRIC, "workload": args.workload, "n_gpus": 1, "unit": UNIT, "higher_is_better": True,
            "data": "synthetic noise windows (timing; injected sources do not change the work)",
            "windows": len(wl.windows), "evals_per_launch": n,
            "mixed": {"value": n / ms_mx * 1e3, "ms": ms_mx, "autotune": tune},
            "fp64": {"value": n / ms_64 * 1e3, "ms": ms_64},
            "mixed_vs_fp64": {"max_abs_dlogL": float(dl.max()), "median_abs_dlogL": float(dl.median())},
            "l2": "flushed between timed launches"}
    # algorithmic rate of the mixed launch (preparation + likelihood kernels)
    f_mid = np.array([w[0] + w[1] / 2 for w in wl.windows]) / wl.T
    flops = sum(w[5] * flops_per_eval(w[2], f, wl.T) for w, f in zip(wl.windows, f_mid))
    peak = 152 * 128 * 2 * 2070e6 / 1e12
    line["mixed"]["roofline"] = {"bound": "alu", "achieved": flops / (ms_mx / 1e3) / 1e12, "peak": peak,
                                 "unit": "TFLOP/s", "frac": flops / (ms_mx / 1e3) / 1e12 / peak,
                                 "kernel": "loglik_mixed_kernel"}
    if args.workload == "band":
        Ns = np.array([w[2] for w in wl.windows])
        per = {}
        for N in np.unique(Ns):
            sub = [w for w in wl.windows if w[2] == N]
            cnt = sum(w[5] for w in sub)
            ms = timed(lambda: ctx.loglik(sub, *data, theta, prec="mixed"), 3)
            per[int(N)] = {"evals": int(cnt), "ms": ms, "evals_per_s": cnt / ms * 1e3}
        line["mixed_by_N"] = per
        # the paper's channel rule: T joins A and E in the windows above f*/2 (Sec. II)
        nT, wT = wk.t_noise_and_weights(wl.windows, wl.T, np.random.default_rng(wk.SEED_BASE + 33))
        dT, wTt = T_(nT, torch.complex128), T_(wT, torch.float64)
        aet = lambda p: ctx.loglik_aet(wl.windows, data[0], data[1], dT, data[2], data[3], wTt, theta, prec=p)
        ms_aet = timed(lambda: aet("mixed"), reps)
        fstar_half = 2.99792458e8 / (4 * np.pi * 2.5e9)
        with_t = [w for w in wl.windows if w[0] / wl.T >= fstar_half]
        l64t = aet("fp64")[0] if n <= 10 ** 6 else None
        line["mixed_aet"] = {"value": n / ms_aet * 1e3, "ms": ms_aet, "windows_with_T": len(with_t),
                             "evals_with_T": int(sum(w[5] for w in with_t)),
                             "rule": "A, E and T in windows whose lowest frequency is at least f*/2 = 9.54 mHz"}
        if l64t is not None:
            line["mixed_aet"]["max_abs_dlogL_vs_fp64"] = float((aet("mixed")[0] - l64t).abs().max())
    if args.workload == "population":
        ms_g = timed(lambda: ctx.loglik_grad(wl.windows, *data, theta, prec="mixed"), reps)
        sub = [(k0, W, N, doff, coff, 512) for (k0, W, N, doff, coff, nc) in wl.windows]
        ms_g64 = timed(lambda: ctx.loglik_grad(sub, *data, theta, prec="fp64"), 1)
        line["grad_mixed"] = {"value": n / ms_g * 1e3, "unit": "gradients/s", "ms": ms_g}
        f_mid = np.array([w[0] + w[1] / 2 for w in wl.windows]) / wl.T
        gflops = sum(w[5] * flops_per_grad(w[2], f, wl.T) for w, f in zip(wl.windows, f_mid))
        peak = 152 * 128 * 2 * 2070e6 / 1e12
        line["grad_mixed"]["roofline"] = {
            "bound": "alu", "achieved": gflops / (ms_g / 1e3) / 1e12, "peak": peak, "unit": "TFLOP/s",
            "frac": gflops / (ms_g / 1e3) / 1e12 / peak, "traffic": profiled_traffic("grad_mixed_population"),
            "kernel": "grad_mixed_kernel",
            "peak_note": "FP32 FMA peak from unit counts: 152 SM x 128 lanes x 2 x 2070 MHz; the timed call "
                         "is the preparation kernel and the gradient kernel"}
        gflops64 = sum(512 * flops_per_grad_fp64(w[2], f, wl.T) for w, f in zip(wl.windows, f_mid))
        line["grad_fp64"] = {"value": 512 * len(sub) / ms_g64 * 1e3, "unit": "gradients/s", "ms": ms_g64,
                             "sample": "512 candidates per window",
                             "roofline": {"bound": "alu", "achieved": gflops64 / (ms_g64 / 1e3) / 1e12,
                                          "peak": fp64_peak_tflops(), "unit": "TFLOP/s",
                                          "frac": gflops64 / (ms_g64 / 1e3) / 1e12 / fp64_peak_tflops(),
                                          "traffic": profiled_traffic("grad_fp64_population"),
                                          "kernel": "grad64_kernel",
                                          "peak_note": "FP64 peak from unit counts: 152 SM x 2 FP64 FMA lanes x 2 "
                                                       "x 2070 MHz; achieved counts the reverse-mode work"}}
        boxes = np.array([np.concatenate([wl.theta[c:c + m].min(0), wl.theta[c:c + m].max(0)])
                          for (_, _, _, _, c, m) in wl.windows])
        ga_ms = {}
        for graph in (False, True):
            ga = GASearch(ctx, wl.windows, *data, boxes, pop=4096, seed=5)
            ga.run(4, graph=graph)
            ga_ms["graph" if graph else "eager"] = timed(lambda: ga.run(200, graph=graph), 1, warm=0,
                                                         flush_l2=False) / 200
        line["ga_generation_ms"] = ga_ms
        line["ga"] = "64 windows x 4,096, gradient-polished elites, 200 generations per timed call"
    line["clocks"] = clocks.stop()
    print(json.dumps(line), flush=True)


def run_fullband(args):
    """Config 5: 0.3-15 mHz at T = 2 yr with the requested number of injected
    binaries, windows from Alg. 1, GA search-and-subtract rounds in every
    window, a 10,000-proposal posterior for every recovered source."""
    from paper_2307_03763_gb300 import api, build, fullband
    build.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    ctx = api.Context(2 * wk.YEAR)
    clocks = ClockSampler(dev.index)
    clocks.start()
    st = fullband.run(ctx, n_src=args.fb_sources, rounds=args.fb_rounds, pop=args.fb_pop, generations=args.fb_gens,
                      phase=not args.fb_no_phase, posterior=args.fb_posterior, scheme=args.fb_scheme,
                      noise=args.fb_noise, joint=not args.fb_no_joint, amp=args.fb_amp,
                      t_short=[float(x) * wk.YEAR for x in args.fb_short.split(",") if float(x) > 0] or None)
    line = {"metric": "total wall time, s per posterior (full-band search)", "workload": "fullband",
            "n_gpus": 1, "unit": "s", "higher_is_better": False, "data": "synthetic",
            "value": st["wall_s"], "s_per_posterior": st["s_per_posterior"],
            "posterior": "Alg. 4: six temperatures (15..1) x 10,000 proposals per recovered source (%s)" % (
                "uniform reduced box, then paired 2-D KDEs" if args.fb_posterior == "kde" else "Gaussian refits"),
            "config": {"workload": "fullband: 0.3-15 mHz, T=2 yr, dt=15 s, %d binaries (%s amplitudes), Alg. 1 "
                                   "windows" % (args.fb_sources, args.fb_amp)}, "stats": st,
            # kernels launched from the host; the GA generations replayed from CUDA graphs are not counted
            "host_kernel_launches": ctx.launch_count(),
            "clocks": clocks.stop()}
    print(json.dumps(line, default=float), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--fp64-steps", type=int, default=None, help="timed steps of the FP64 path (default: steps)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-graph", action="store_true", help="time the steps with eager launches, not graph replays")
    ap.add_argument("--shard", action="store_true",
                    help="under torchrun: share the 16 windows out among the ranks (strong scaling) instead of "
                         "one replica of the workload per rank (weak scaling)")
    ap.add_argument("--workload", default="posterior", choices=["posterior", "tiny", "band", "population", "fullband"],
                    help="posterior: the headline step; the others print their own figures")
    ap.add_argument("--fb-sources", type=int, default=200000, help="fullband: injected binaries")
    ap.add_argument("--fb-rounds", type=int, default=3, help="fullband: search-and-subtract rounds")
    ap.add_argument("--fb-pop", type=int, default=1024, help="fullband: GA population per window")
    ap.add_argument("--fb-gens", type=int, default=100, help="fullband: GA generations per round")
    ap.add_argument("--fb-scheme", default="all", choices=["all", "evenodd"],
                    help="fullband: all windows at once, or the paper's even/odd runs (Table 2)")
    ap.add_argument("--fb-noise", default="true", choices=["true", "median"],
                    help="fullband: weights from the true PSD, or each segment's median periodogram")
    ap.add_argument("--fb-posterior", default="gauss", choices=["gauss", "kde"],
                    help="fullband: Alg. 4 proposals, Gaussian refits or the paper's paired KDEs")
    ap.add_argument("--fb-no-joint", action="store_true",
                    help="fullband: no joint refit of a window's sources after each new one (Alg. 2)")
    ap.add_argument("--fb-amp", default="loguniform", choices=["loguniform", "galactic"],
                    help="fullband: amplitudes log-uniform on [1e-23, 1e-21] (the workload's) or N(>A) ~ A^-2 "
                         "(about a tenth of the sources loud)")
    ap.add_argument("--fb-short", default="0.5,1",
                    help="fullband: years of shorter observations searched first, comma-separated, each seeding "
                         "the next and the last the full one (Sec. III.E); 0 for none")
    ap.add_argument("--fb-no-phase", action="store_true",
                    help="fullband: rank GA individuals by the plain SNR instead of the SNR maximised over phi0")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.workload == "fullband":
        return run_fullband(args)
    if args.workload != "posterior":
        return run_workload(args)

    from paper_2307_03763_gb300 import api, build
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    build.build()
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    ctx = api.Context(2 * wk.YEAR, device=dev.index)
    shard = args.shard and world > 1
    wl, dA_h, dE_h, th_h, lg_h = build_inputs(ctx, wk.SEED_BASE + 2 + (0 if shard else 1000 * rank), dev)
    n_total = wl.n_cand
    if shard:
        # strong scaling: every rank builds the same windows and keeps its
        # cost-balanced share (no exchange on the data path)
        import dataclasses
        from paper_2307_03763_gb300 import shard as sh
        part = sh.Shard(wl.windows, world, rank)
        if not part.windows:
            raise SystemExit("--shard: more ranks than windows")
        dA_h, dE_h, wA_h, wE_h = part.take_data(dA_h, dE_h, wl.w_A, wl.w_E)
        th_h, lg_h = part.take_candidates(th_h), part.take_candidates(lg_h)
        meta = dict(wl.meta)
        for key in ("source", "fisher_sigma"):
            meta[key] = np.asarray(wl.meta[key])[part.window_ids]
        wl = dataclasses.replace(wl, windows=part.windows, w_A=wA_h, w_E=wE_h, theta=th_h,
                                 log_u=part.take_candidates(wl.log_u), noise_A=dA_h, noise_E=dE_h, meta=meta)
    nwin, n = len(wl.windows), wl.windows[0][5]
    T_ = lambda x, dt: torch.as_tensor(np.ascontiguousarray(x)).to(dev, dt)
    dA, dE = T_(dA_h, torch.complex128), T_(dE_h, torch.complex128)
    wA, wE = T_(wl.w_A, torch.float64), T_(wl.w_E, torch.float64)
    theta = T_(th_h, torch.float64)
    log_g = T_(lg_h.reshape(nwin, n), torch.float64)
    log_u = T_(wl.log_u.reshape(nwin, n), torch.float64)
    temp = torch.ones(nwin, dtype=torch.float64, device=dev)
    logL = torch.empty(wl.n_cand, dtype=torch.float64, device=dev)
    chain = torch.empty((nwin, n), dtype=torch.int32, device=dev)
    acc = torch.empty(nwin, dtype=torch.int32, device=dev)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    # certified rounds: per proposal the mixed logL, <d|h>, <h|h>; per chain the
    # rows re-evaluated in FP64; one "pending" word per call (0: certified)
    dh_b = torch.empty_like(logL)
    hh_b = torch.empty_like(logL)
    n_slots = max(args.steps, args.warmup, 8) + 1
    pend = torch.zeros(n_slots, dtype=torch.int32, device=dev)
    n_exact = torch.zeros((n_slots, nwin), dtype=torch.int32, device=dev)

    def certified(k=0):
        ctx.mh_certified(wl.windows, dA, dE, wA, wE, theta, log_g, log_u, temp, max_iter=MAX_ITER,
                         out=(chain, acc, logL, dh_b, hh_b, n_exact[k], pend[k:k + 1]))

    def step(prec):
        if prec == "certified":
            return certified()
        ctx.loglik(wl.windows, dA, dE, wA, wE, theta, prec=prec, out=(logL, None, None))
        ctx.mh_independence(logL.view(nwin, n), log_g, log_u, temp, out=(chain, acc))

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)

    pmax = torch.zeros(1, dtype=torch.int32, device=dev)

    def captured(prec):
        """One step of `prec` captured in a CUDA graph (after eager warm-up
        calls that size the library's scratch), and the library kernels it
        launches.  The certified step also folds its pending word into a
        running maximum, so that every replay's certification is checked."""
        side = torch.cuda.Stream(dev)
        side.wait_stream(stream)
        with torch.cuda.stream(side):
            for _ in range(2):
                step(prec)
        stream.wait_stream(side)
        torch.cuda.synchronize(dev)
        g = torch.cuda.CUDAGraph()
        n0 = ctx.launch_count()
        with torch.cuda.graph(g, stream=side):
            if prec == "certified":
                certified(0)
                torch.maximum(pmax, pend[0:1], out=pmax)
            else:
                step(prec)
        torch.cuda.synchronize(dev)
        return g, ctx.launch_count() - n0

    def timed(prec, steps, graph=False):
        """Per-step CUDA-event times (ms) of the step and, for the plain
        precisions run eagerly, of the likelihood launch alone."""
        g = None
        if graph:
            g, per_step = captured(prec)
        for _ in range(args.warmup):
            g.replay() if g is not None else step(prec)
        barrier()
        st = []
        n0 = ctx.launch_count()
        torch.cuda.nvtx.range_push(f"timed_{prec}")   # lets a profiler select the timed launches
        kev = []
        for k in range(steps):
            flush.zero_()                      # L2 flush between timed steps
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            if g is None and prec == "mixed":
                # the library records these around the likelihood kernels alone
                k0, k1 = (torch.cuda.Event(enable_timing=True) for _ in range(2))
                k0.record(stream)
                k1.record(stream)
                ctx.set_kernel_events(k0, k1)
                kev.append((k0, k1))
            e0.record(stream)
            if g is not None:
                g.replay()
                e1.record(stream)
            elif prec == "certified":
                certified(k)
                e1.record(stream)
            else:
                ctx.loglik(wl.windows, dA, dE, wA, wE, theta, prec=prec, out=(logL, None, None))
                e1.record(stream)
                ctx.mh_independence(logL.view(nwin, n), log_g, log_u, temp, out=(chain, acc))
            e2.record(stream)
            st.append((e0, e1, e2))
        torch.cuda.nvtx.range_pop()
        launches = per_step * steps if g is not None else ctx.launch_count() - n0
        barrier()
        step_ms = [a.elapsed_time(c) for a, b, c in st]
        kern_ms = [a.elapsed_time(b) for a, b, c in st]
        if kev:
            timed.kernel_only_ms = float(np.mean([a.elapsed_time(b) for a, b in kev]))
        return float(np.sum(step_ms)), float(np.mean(kern_ms)), launches

    def max_over_ranks(x):
        if world == 1:
            return x
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        return float(t.item())

    # launch shapes for this batch from the library's autotuner (untimed)
    tuning = {p: ctx.autotune(wl.windows, dA, dE, wA, wE, theta, prec=p, reps=3) for p in ("mixed", "fp64")}

    # accuracy of the mixed path against the FP64 path on this workload, and
    # the certified chains against the chains of the FP64 path (untimed)
    l64, dh64, hh64 = (torch.empty_like(logL) for _ in range(3))
    ctx.loglik(wl.windows, dA, dE, wA, wE, theta, prec="fp64", out=(l64, dh64, hh64))
    lmx = torch.empty_like(logL)
    ctx.loglik(wl.windows, dA, dE, wA, wE, theta, prec="mixed", out=(lmx, None, None))
    ch64, acc64 = ctx.mh_independence(l64.view(nwin, n), log_g, log_u, temp)
    certified()
    torch.cuda.synchronize(dev)
    chains_equal = bool(torch.equal(chain, ch64)) and bool(torch.equal(acc, acc64)) and int(pend[0]) == 0
    redo = logL != lmx
    rows_equal = bool(torch.equal(logL[redo], l64[redo]))
    dl = (lmx - l64).abs()
    snr = hh64.clamp(min=0).sqrt()
    by_snr = {}
    for lo, hi in [(0, 20), (20, 50), (50, 100), (100, 200), (200, None)]:
        m = (snr >= lo) if hi is None else (snr >= lo) & (snr < hi)
        if bool(m.any()):
            by_snr["%d-%s" % (lo, hi if hi else "")] = {
                "proposals": int(m.sum()), "max_abs_dlogL": float(dl[m].max()),
                "p99_abs_dlogL": float(dl[m].quantile(0.99)), "median_abs_dlogL": float(dl[m].median())}
    ctx.check()

    # clocks sampled over the timed regions (each alone can be shorter than
    # the sampling interval)
    clocks = ClockSampler(dev.index)
    clocks.start()
    graphs = not args.no_graph
    pmax.zero_()
    tot_c, _, launches_c = timed("certified", args.steps, graph=graphs)
    pend_max = int(pmax.item()) if graphs else int(pend[:args.steps].max())
    exact_rows = n_exact[:1].sum(1).double() if graphs else n_exact[:args.steps].sum(1).double()
    tot_mxg, _, _ = timed("mixed", args.steps, graph=graphs)
    tot_mx, kern_mx, _ = timed("mixed", args.steps)          # eager: the likelihood call's own events
    kern_only_mx = max_over_ranks(timed.kernel_only_ms)      # the likelihood kernel alone (library events)
    fp64_steps = args.fp64_steps or max(3, args.steps // 10)
    tot_64, kern_64, _ = timed("fp64", fp64_steps)
    clk = clocks.stop()
    tot_c, tot_mx, tot_mxg, tot_64 = (max_over_ranks(x) for x in (tot_c, tot_mx, tot_mxg, tot_64))

    # end to end through the public API with host buffers: proposals and their
    # log g, log u (and the window data) copied in from pinned memory each
    # step, chain and logL copied out.  Two buffer sets and a copy stream
    # overlap step k's copies with the compute of its neighbours; every byte
    # of every step still crosses the link inside the timed region.
    pin = lambda x: torch.as_tensor(np.ascontiguousarray(x)).pin_memory()
    h_in = [pin(th_h), pin(lg_h.reshape(nwin, n)), pin(wl.log_u.reshape(nwin, n)), pin(dA_h), pin(dE_h),
            pin(wl.w_A), pin(wl.w_E)]
    h_out = [(torch.empty((nwin, n), dtype=torch.int32).pin_memory(),
              torch.empty(wl.n_cand, dtype=torch.float64).pin_memory()) for _ in range(2)]
    d_in = [[torch.empty_like(x, device=dev) for x in h_in] for _ in range(2)]
    d_out = [(torch.empty((nwin, n), dtype=torch.int32, device=dev),
              torch.empty(nwin, dtype=torch.int32, device=dev),
              torch.empty(wl.n_cand, dtype=torch.float64, device=dev),
              torch.empty(wl.n_cand, dtype=torch.float64, device=dev),
              torch.empty(wl.n_cand, dtype=torch.float64, device=dev),
              torch.empty(nwin, dtype=torch.int32, device=dev),
              torch.empty(1, dtype=torch.int32, device=dev)) for _ in range(2)]
    h2d = sum(h.numel() * h.element_size() for h in h_in)
    d2h = h_out[0][0].numel() * 4 + h_out[0][1].numel() * 8
    copy = torch.cuda.Stream(dev)
    ev_in = [torch.cuda.Event() for _ in range(2)]
    ev_comp = [torch.cuda.Event() for _ in range(2)]
    ev_free = [torch.cuda.Event() for _ in range(2)]
    for e in ev_free:
        e.record(copy)

    def e2e_h2d(k):
        b = k % 2
        with torch.cuda.stream(copy):
            copy.wait_event(ev_free[b])            # the buffer's previous outputs have left
            for h, d in zip(h_in, d_in[b]):
                d.copy_(h, non_blocking=True)
            ev_in[b].record(copy)

    def e2e_call(b):
        th_d, lg_d, lu_d, dA_d, dE_d, wA_d, wE_d = d_in[b]
        ctx.mh_certified(wl.windows, dA_d, dE_d, wA_d, wE_d, th_d, lg_d, lu_d, temp, max_iter=MAX_ITER,
                         out=d_out[b])

    # gb_mh_certified can be captured: unless --no-graph, each buffer set's
    # call is captured once (on real inputs, after eager calls that size the
    # library's scratch) and every step replays it
    e2e_graphs = None
    if not args.no_graph:
        e2e_graphs = []
        side = torch.cuda.Stream(dev)
        for b in range(2):
            for h, d in zip(h_in, d_in[b]):
                d.copy_(h)
            side.wait_stream(stream)
            with torch.cuda.stream(side):
                e2e_call(b)
                e2e_call(b)
            stream.wait_stream(side)
            torch.cuda.synchronize(dev)
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=side):
                e2e_call(b)
            e2e_graphs.append(g)
        torch.cuda.synchronize(dev)

    def e2e_compute(k):
        b = k % 2
        stream.wait_event(ev_in[b])
        if e2e_graphs is not None:
            with torch.cuda.stream(stream):
                e2e_graphs[b].replay()
        else:
            e2e_call(b)
        ev_comp[b].record(stream)

    def e2e_d2h(k):
        b = k % 2
        with torch.cuda.stream(copy):
            copy.wait_event(ev_comp[b])
            h_out[b][0].copy_(d_out[b][0], non_blocking=True)
            h_out[b][1].copy_(d_out[b][2], non_blocking=True)
            ev_free[b].record(copy)

    def e2e_run(steps):
        e2e_h2d(0)
        for k in range(steps):
            if k + 1 < steps:
                e2e_h2d(k + 1)
            e2e_compute(k)
            e2e_d2h(k)

    e2e_run(args.warmup)
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(copy)
    e2e_run(args.steps)
    e1.record(copy)
    barrier()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1))
    # the outputs of the last step equal a device-resident certified step's (untimed)
    certified()
    torch.cuda.synchronize(dev)
    assert torch.equal(h_out[(args.steps - 1) % 2][0], chain.cpu())
    assert torch.equal(h_out[(args.steps - 1) % 2][1], logL.cpu())

    if rank != 0:
        return
    evals = n_total if shard else wl.n_cand * world
    value = evals * args.steps / (tot_c / 1e3)
    value_mx = evals * args.steps / (tot_mxg / 1e3)
    value64 = evals * fp64_steps / (tot_64 / 1e3)
    ms_step = tot_c / args.steps
    f_mid = np.array([w[0] + w[1] / 2 for w in wl.windows]) / wl.T
    flops = sum(n * flops_per_eval(w[2], f, wl.T) for w, f in zip(wl.windows, f_mid))
    flops64 = sum(n * flops_per_eval_fp64(w[2], f, wl.T) for w, f in zip(wl.windows, f_mid))
    fp32_peak = 152 * 128 * 2 * 2070e6 / 1e12
    achieved = flops / (kern_only_mx / 1e3) / 1e12
    achieved64 = flops64 / (kern_64 / 1e3) / 1e12
    # Alg. 4 with its temperature ladder (15, 10, 5, 3, 2, 1): six rounds of
    # 10,000 device-drawn proposals per window, Gaussian refits between rounds
    from paper_2307_03763_gb300.posterior import AnnealedPosterior
    sig = wl.meta["fisher_sigma"]
    # start: the T = 15 tempered Fisher width, widened by 1.2
    cov = np.stack([np.diag(15.0 * (1.2 * sig[w]) ** 2) for w in range(nwin)])
    ap = AnnealedPosterior(ctx, wl.windows, dA, dE, wA, wE, wl.meta["source"], cov, n, seed=11)
    ap.run(graph=True)                    # eager ladder, then the capture
    ann_ms = []
    for rep in range(5):                  # each replay: a new posterior from the initial proposal
        barrier()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        ap.run(graph=True)
        a1.record(stream)
        barrier()
        ann_ms.append(a0.elapsed_time(a1))
    ann_ms = max_over_ranks(float(np.median(ann_ms)))
    annealed = {"s_per_posterior": ann_ms / 1e3 / nwin, "temperatures": ap.temperatures,
                "proposals_per_round": n, "windows": nwin, "ms_per_batch": ann_ms,
                "accept_rate_T1_median": float((ap.rounds.accepted.float() / n).median()),
                "proposal_refit": "Gaussian of the visited states on the device (the paper refits 2-D KDEs)",
                "graph": "the six rounds and five refits replayed from one CUDA graph"}
    # the same ladder with the paper's proposals: uniform over the reduced box
    # (MLE +- 4 sigma, f0 +- sigma, fdot over its prior, narrow psi and phi0),
    # then paired 2-D KDEs of each temperature's chain
    from paper_2307_03763_gb300.posterior import KDEPosterior, reduced_box
    f_lo = np.array([w[0] / wl.T for w in wl.windows])
    f_hi = np.array([(w[0] + w[1]) / wl.T for w in wl.windows])
    plo = np.stack([np.array([a, 0.0, -np.pi / 2, -np.pi, 1e-24, 0.0, 0.0, 0.0]) for a in f_lo])
    phi = np.stack([np.array([b, float(wk.chirp_fdot(b, 1.0)), np.pi / 2, np.pi, 1e-20, np.pi, np.pi, 2 * np.pi])
                    for b in f_hi])
    kp = KDEPosterior(ctx, wl.windows, dA, dE, wA, wE, reduced_box(wl.meta["source"], sig, plo, phi), n, seed=12)
    kp.run(graph=True)
    kde_ms = []
    for rep in range(5):
        barrier()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        kp.run(graph=True)
        a1.record(stream)
        barrier()
        kde_ms.append(a0.elapsed_time(a1))
    kde_ms = max_over_ranks(float(np.median(kde_ms)))
    annealed_kde = {"s_per_posterior": kde_ms / 1e3 / nwin, "temperatures": kp.temperatures,
                    "proposals_per_round": n, "windows": nwin, "ms_per_batch": kde_ms,
                    "accept_rate_T1_median": float((kp.accepted.float() / n).median()),
                    "proposal": "uniform over the reduced box, then paired 2-D grid KDEs (f0-fdot, lambda-beta, "
                                "A-iota; %d x %d cells) of each temperature's chain" % (kp.grid, kp.grid),
                    "graph": "the six rounds and five KDE builds replayed from one CUDA graph"}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "strong" if shard else "weak",
        "vs_baseline": None, "dtype": "f32+f64-phase", "data": "synthetic",
        "config": {"workload": WORKLOAD, "global_batch": evals, "windows": nwin, "proposals_per_window": n,
                   "l2": "flushed between timed steps (2x L2 buffer written)",
                   "parallelism": ("windows sharded over %d ranks (cost-balanced)" % world) if shard else
                                  "replicas" if world > 1 else "single GPU",
                   "launch": "each timed step replayed from a CUDA graph" if graphs else "eager launches",
                   "step": "gb_mh_certified: mixed-precision logL of every proposal, the chains, FP64 "
                           "re-evaluation of the proposals whose decision the mixed error bound cannot settle"},
        "s_per_10k_posterior": ms_step / 1e3 / nwin,
        "certified": {"chains_equal_fp64_chains": chains_equal, "reevaluated_rows_equal_fp64": rows_equal,
                      "eps": api.MIXED_EPS, "max_iter": MAX_ITER, "pending_max_over_steps": pend_max,
                      "rows_reevaluated_per_step": float(exact_rows.mean()),
                      "reevaluated_fraction": float(exact_rows.mean()) / evals,
                      "added_ms_per_step": ms_step - tot_mxg / args.steps},
        "mixed_uncertified": {"value": value_mx, "unit": UNIT, "ms_per_step": tot_mxg / args.steps,
                              "eager_ms_per_step": tot_mx / args.steps,
                              "loglik_ms": kern_mx, "loglik_kernel_ms": kern_only_mx,
                              "mh_ms": tot_mx / args.steps - kern_mx,
                              "s_per_10k_posterior": tot_mxg / args.steps / 1e3 / nwin},
        "annealed_posterior_6T": annealed,
        "annealed_posterior_6T_kde": annealed_kde,
        "fp64": {"value": value64, "unit": UNIT, "steps": fp64_steps, "ms_per_step": tot_64 / fp64_steps,
                 "s_per_10k_posterior": tot_64 / fp64_steps / 1e3 / nwin, "loglik_ms": kern_64,
                 "roofline": {"bound": "alu", "achieved": achieved64, "peak": fp64_peak_tflops(),
                              "unit": "TFLOP/s", "frac": achieved64 / fp64_peak_tflops(),
                              "traffic": profiled_traffic("loglik_fp64_posterior"),
                              "kernel": "loglik64_kernel",
                              "peak_note": "FP64 peak from unit counts: 152 SM x 2 FP64 FMA lanes x 2 x 2070 MHz "
                                           "(the nominal 1.25 TFLOP/s dense FP64)"}},
        "mixed_vs_fp64": {"max_abs_dlogL": float(dl.max()), "p99_abs_dlogL": float(dl.quantile(0.99)),
                          "median_abs_dlogL": float(dl.median()), "snr_range": [20, 200],
                          "by_proposal_snr": by_snr},
        "loglik_ms": kern_mx,
        "autotune": tuning,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                     "frac": achieved / fp32_peak, "traffic": profiled_traffic(),
                     "kernel": "loglik_mixed_kernel",
                     "kernel_ms": kern_only_mx,
                     "peak_note": "FP32 FMA peak from unit counts: 152 SM x 128 lanes x 2 x 2070 MHz; achieved "
                                  "from the likelihood kernel's own duration in the uncertified eager steps "
                                  "(events the library records around it, after the window preparation)"},
        "e2e": {"value": evals * args.steps / (e2e_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h,
                "launch": "eager calls" if args.no_graph else "the certified call replayed from a CUDA graph per "
                                                              "buffer set; copies on a second stream"},
        "clocks": clk,
        # library kernels launched in the timed certified steps, counted by the
        # context (window preparation, likelihood, chains, bounds,
        # certification passes, FP64 re-evaluation and flip checks)
        "gpu_launches": launches_c,
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"], line["cpu_baseline_fft"] = cpu_baseline(wl, dA_h, dE_h, th_h)
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
