"""Seeded synthetic inputs for the Galactic-binary likelihood path.

This module holds none of the likelihood arithmetic: it draws source
parameters, window layouts, candidate batches, proposal variates and detector
noise, and evaluates the analytic noise PSD those draws need.  The template
that a source adds to the data is *not* computed here; callers inject it with
whichever implementation they are exercising.  Nothing here imports torch or
the CUDA library, so every consumer can use it.

Workloads follow the paper's data shapes (Sec. IV: 0.3 mHz up to Nyquist,
dt = 15 s, T_obs = 0.5-2 yr, many overlapping Galactic binaries); the LDC data
sets the paper analyses are not available, so these draws stand in for them.
"""
import dataclasses
import math

import numpy as np

YEAR = 31557600.0
C_LIGHT = 299792458.0
ARM_L = 2.5e9
DT_SAMPLE = 15.0
G_MSUN_S = 4.925490947641267e-06   # G M_sun / c^3 in seconds
SEED_BASE = 230703763

PARAM_NAMES = ("f0", "fdot", "beta", "lam", "A", "iota", "psi", "phi0")


# ----------------------------------------------------------------------------
# noise model and physical scalings used to shape the draws
# ----------------------------------------------------------------------------

def psd_AE(f, L=ARM_L):
    """One-sided analytic PSD of TDI A (= E), fractional-frequency units.

    Test-mass acceleration 3e-15 m/s^2/rtHz with the usual low/high-frequency
    shaping, optical metrology 15e-12 m/rtHz, first-generation A/E transfer,
    x = 2 pi f L / c:
      S_acc = (3e-15)^2 (1 + (0.4 mHz/f)^2)(1 + (f/8 mHz)^4) / (2 pi f c)^2
      S_oms = (15e-12)^2 (1 + (2 mHz/f)^4) (2 pi f / c)^2
      S_A   = 8 sin^2 x [(2 + cos x) S_oms + 2 (3 + 2 cos x + cos 2x) S_acc]
    """
    f = np.asarray(f, dtype=np.float64)
    x = 2.0 * np.pi * f * L / C_LIGHT
    s_acc = (3e-15) ** 2 * (1 + (0.4e-3 / f) ** 2) * (1 + (f / 8e-3) ** 4) / (2 * np.pi * f * C_LIGHT) ** 2
    s_oms = (15e-12) ** 2 * (1 + (2e-3 / f) ** 4) * (2 * np.pi * f / C_LIGHT) ** 2
    return 8.0 * np.sin(x) ** 2 * ((2 + np.cos(x)) * s_oms + 2 * (3 + 2 * np.cos(x) + np.cos(2 * x)) * s_acc)


def psd_T(f, L=ARM_L):
    """One-sided analytic PSD of TDI T for the same two noises and the
    first-generation T transfer, x = 2 pi f L / c:
      S_T = 16 sin^2 x [(1 - cos x) S_oms + 2 (1 - cos x)^2 S_acc]."""
    f = np.asarray(f, dtype=np.float64)
    x = 2.0 * np.pi * f * L / C_LIGHT
    s_acc = (3e-15) ** 2 * (1 + (0.4e-3 / f) ** 2) * (1 + (f / 8e-3) ** 4) / (2 * np.pi * f * C_LIGHT) ** 2
    s_oms = (15e-12) ** 2 * (1 + (2e-3 / f) ** 4) * (2 * np.pi * f / C_LIGHT) ** 2
    return 16.0 * np.sin(x) ** 2 * ((1 - np.cos(x)) * s_oms + 2 * (1 - np.cos(x)) ** 2 * s_acc)


def t_noise_and_weights(windows, T, rng):
    """T-channel noise, Re and Im ~ N(0, T S_T / 4) per bin, and w = 1/S_T."""
    nb = sum(w[1] for w in windows)
    nT = np.empty(nb, np.complex128)
    wT = np.empty(nb)
    for (k0, W, N, doff, _, _) in windows:
        S = psd_T((k0 + np.arange(W)) / T)
        nT[doff:doff + W] = np.sqrt(T * S / 4.0) * (rng.standard_normal(W) + 1j * rng.standard_normal(W))
        wT[doff:doff + W] = 1.0 / S
    return nT, wT


def chirp_fdot(f, mchirp_msun):
    """fdot = 96/5 pi^(8/3) Mc^(5/3) f^(11/3) in geometric units (Eq. 8)."""
    mc = np.asarray(mchirp_msun, dtype=np.float64) * G_MSUN_S
    return 96.0 / 5.0 * np.pi ** (8.0 / 3.0) * mc ** (5.0 / 3.0) * np.asarray(f, dtype=np.float64) ** (11.0 / 3.0)


def bandwidth_max(f, T, mchirp_msun=None):
    """Broadest expected signal B_max = B_F + 2 B_O + 2 B_C in Hz (Sec. III.A).

    B_F = fdot_max T with fdot_max from Eq. 8 (Chandrasekhar-mass binary by
    default, Mc = (1.4*1.4)^(3/5)/2.8^(1/5) M_sun), B_O = 1e-4 f, B_C = 4/yr.
    """
    if mchirp_msun is None:
        mchirp_msun = (1.4 * 1.4) ** 0.6 / (2.8) ** 0.2
    return chirp_fdot(f, mchirp_msun) * T + 2e-4 * np.asarray(f) + 8.0 / YEAR


def segments(f_min, f_max, T):
    """Frequency segments [f, f + 2 B_max(f)) from f_min to f_max (Alg. 1)."""
    out = []
    f = f_min
    while f < f_max:
        f_next = f + 2.0 * float(bandwidth_max(f, T))
        out.append((f, f_next))
        f = f_next
    return out


def n_for_band(f, T, mchirp_max=1.0):
    """Smallest power of two >= 2 B_max(f) T bins (with the given chirp-mass cap)."""
    bins = 2.0 * float(bandwidth_max(f, T, mchirp_max)) * T
    return 1 << max(5, int(math.ceil(math.log2(bins))))


# ----------------------------------------------------------------------------
# workload container
# ----------------------------------------------------------------------------

@dataclasses.dataclass
class Workload:
    """Host-side description of one batch.

    windows: list of (k0, W, N, data_off, cand_off, n_cand) -- the layout the
    library's window descriptor uses.  noise_A/E: complex128 noise on all window
    bins, concatenated; w_A/E: 1/S per bin; sources: list (per window) of (8,)
    parameter arrays to inject; theta: (n_total, 8) candidates; log_g: proposal
    log-density per candidate (or None); log_u: log of U(0,1) per candidate.
    """
    name: str
    T: float
    windows: list
    noise_A: np.ndarray
    noise_E: np.ndarray
    w_A: np.ndarray
    w_E: np.ndarray
    sources: list
    theta: np.ndarray
    log_g: np.ndarray = None
    log_u: np.ndarray = None
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def n_cand(self):
        return int(self.theta.shape[0])

    @property
    def n_bins(self):
        return int(self.w_A.shape[0])


def random_angles(rng, n):
    """beta, lambda, iota, psi, phi0 uniform on the prior ranges of Table 1."""
    beta = np.arcsin(rng.uniform(-1.0, 1.0, n))
    lam = rng.uniform(-np.pi, np.pi, n)
    iota = np.arccos(rng.uniform(-1.0, 1.0, n))
    psi = rng.uniform(0.0, np.pi, n)
    phi0 = rng.uniform(0.0, 2.0 * np.pi, n)
    return beta, lam, iota, psi, phi0


def source(f0, fdot, A, rng):
    beta, lam, iota, psi, phi0 = random_angles(rng, 1)
    return np.array([f0, fdot, beta[0], lam[0], A, iota[0], psi[0], phi0[0]])


def layout(window_specs, counts):
    """Concatenate windows (k0, W, N) with candidate counts into descriptors."""
    wins, doff, coff = [], 0, 0
    for (k0, W, N), nc in zip(window_specs, counts):
        wins.append((int(k0), int(W), int(N), doff, coff, int(nc)))
        doff += W
        coff += nc
    return wins, doff, coff


def noise_and_weights(windows, T, rng):
    """Complex Gaussian noise, Re and Im ~ N(0, T S / 4) per bin, and w = 1/S."""
    nb = sum(w[1] for w in windows)
    nA = np.empty(nb, np.complex128)
    nE = np.empty(nb, np.complex128)
    wA = np.empty(nb)
    for (k0, W, N, doff, _, _) in windows:
        f = (k0 + np.arange(W)) / T
        S = psd_AE(f)
        sd = np.sqrt(T * S / 4.0)
        nA[doff:doff + W] = sd * (rng.standard_normal(W) + 1j * rng.standard_normal(W))
        nE[doff:doff + W] = sd * (rng.standard_normal(W) + 1j * rng.standard_normal(W))
        wA[doff:doff + W] = 1.0 / S
    return nA, nE, wA, wA.copy()


def uniform_box(center, half, n, rng):
    """n draws uniform in center +- half (per parameter)."""
    return center[None, :] + half[None, :] * rng.uniform(-1.0, 1.0, (n, 8))


def gaussian_proposals(mu, sigma, n, rng):
    """n draws ~ N(mu, diag sigma^2) and their log-density log g (independence proposal)."""
    z = rng.standard_normal((n, 8))
    th = mu[None, :] + sigma[None, :] * z
    log_g = -0.5 * (z * z).sum(1) - np.log(sigma).sum() - 4.0 * np.log(2.0 * np.pi)
    return th, log_g


def log_uniforms(n, rng):
    """log u with u ~ U(0, 1) open at 0 (the MH accept variates, passed in as logs)."""
    u = rng.uniform(np.finfo(np.float64).tiny, 1.0, n)
    return np.log(u)


# ----------------------------------------------------------------------------
# the five workloads
# ----------------------------------------------------------------------------

def fullband_sources(n_src=200000, f_lo=0.3e-3, f_hi=15e-3, seed=SEED_BASE + 5, amp="loguniform"):
    """The full-band population: f0 log-uniform in [f_lo, f_hi], fdot from
    Eq. 8 with Mc ~ U[0.2, 1] M_sun, angles on the Table 1 ranges; (n_src, 8),
    sorted by f0.  Amplitudes: "loguniform" (the full-band workload's),
    log-uniform on [1e-23, 1e-21] (at T = 2 yr with the instrument PSD
    134,550 of the 200,000 lie above SNR 10, one per ~7 bins); "galactic",
    a power law N(>A) ~ A^-2 on [4e-24, 1e-21] (a disk population: most
    sources faint, 19,493 above SNR 10, one per ~47 bins, against 18,332
    above SNR 10 in the 2-yr data set of Table 4)."""
    rng = np.random.default_rng(seed)
    f0 = np.sort(np.exp(rng.uniform(np.log(f_lo), np.log(f_hi), n_src)))
    fdot = chirp_fdot(f0, rng.uniform(0.2, 1.0, n_src))
    if amp == "galactic":
        a_lo, a_hi = 4e-24, 1e-21
        u = rng.uniform(0.0, 1.0, n_src)
        A = a_lo / np.sqrt(1.0 - u * (1.0 - (a_lo / a_hi) ** 2))
    elif amp == "loguniform":
        A = np.exp(rng.uniform(np.log(1e-23), np.log(1e-21), n_src))
    else:
        raise ValueError("amp must be 'galactic' or 'loguniform'")
    beta, lam, iota, psi, phi0 = random_angles(rng, n_src)
    return np.stack([f0, fdot, beta, lam, A, iota, psi, phi0], 1)


def fullband_layout(f_lo=0.3e-3, f_hi=15e-3, T=2 * YEAR, n_cap=1024):
    """Search windows from the segments of Alg. 1: [(k0, N, ka, kb)], the
    segment's bins [ka, kb) (the frequency range searched there) and a window
    of N bins centred on it, N the smallest power of two (>= 32) that holds
    the segment.  A segment wider than n_cap bins is split into equal parts."""
    out = []
    for fa, fb in segments(f_lo, f_hi, T):
        ka, kb = int(math.floor(fa * T)), int(math.ceil(fb * T))
        parts = max(1, int(math.ceil((kb - ka) / n_cap)))
        edges = np.linspace(ka, kb, parts + 1).round().astype(np.int64)
        for a, b in zip(edges[:-1], edges[1:]):
            N = 1 << max(5, int(math.ceil(math.log2(max(int(b - a), 1)))))
            c = (int(a) + int(b)) // 2
            out.append((c - N // 2, N, int(a), int(b)))
    return out


def band_noise(k_lo, k_hi, T, rng):
    """Noise on the contiguous bins [k_lo, k_hi): Re, Im ~ N(0, T S / 4), and w = 1/S."""
    f = np.arange(k_lo, k_hi, dtype=np.float64) / T
    S = psd_AE(f)
    sd = np.sqrt(T * S / 4.0)
    n = k_hi - k_lo
    nA = sd * (rng.standard_normal(n) + 1j * rng.standard_normal(n))
    nE = sd * (rng.standard_normal(n) + 1j * rng.standard_normal(n))
    return nA, nE, 1.0 / S

def tiny_window(seed=SEED_BASE + 1, n_cand=1000, N=128, T=2 * YEAR):
    """One window of N = W = 128 bins at f0 = 1.5 mHz, T = 2 yr; 1,000 candidates
    uniform in a box around the injected source (f0 +- 5/T, fdot in [0, 2 fdot],
    angles +- 0.1 rad, A +- 10 %)."""
    rng = np.random.default_rng(seed)
    f0, fdot, A = 1.5e-3, 1e-17, 1e-22
    src = source(f0, fdot, A, rng)
    kc = int(math.floor((f0 + 0.5 * fdot * T) * T + 0.5))
    wins, _, _ = layout([(kc - N // 2, N, N)], [n_cand])
    nA, nE, wA, wE = noise_and_weights(wins, T, rng)
    half = np.array([5.0 / T, fdot, 0.1, 0.1, 0.1 * A, 0.1, 0.1, 0.1])
    th = uniform_box(src, half, n_cand, rng)
    th[:, 2] = np.clip(th[:, 2], -np.pi / 2, np.pi / 2)
    return Workload("tiny: 1 window N=128, f0=1.5 mHz, T=2 yr, 1000 candidates", T, wins,
                    nA, nE, wA, wE, [[src]], th, None, log_uniforms(n_cand, rng),
                    {"seed": seed})


def posterior_windows(seed=SEED_BASE + 2, n_win=16, n_prop=10000, T=2 * YEAR):
    """16 windows, f0 log-uniform in [0.5, 5] mHz, N = 128 below 3.6 mHz else 256,
    one source per window with a target SNR log-uniform in [20, 200].

    Returns the layout, noise and sources at unit amplitude (A = 1) plus the
    target SNRs; the caller rescales A to the SNR and draws the proposals with
    ``gaussian_proposals`` once it knows the Fisher widths.
    """
    rng = np.random.default_rng(seed)
    f0s = np.exp(rng.uniform(np.log(0.5e-3), np.log(5e-3), n_win))
    snr = np.exp(rng.uniform(np.log(20.0), np.log(200.0), n_win))
    specs, srcs = [], []
    for f0 in f0s:
        N = 128 if f0 < 3.6e-3 else 256
        mc = rng.uniform(0.2, 1.0)
        fdot = float(chirp_fdot(f0, mc))
        s = source(f0, fdot, 1.0, rng)
        kc = int(math.floor((f0 + 0.5 * fdot * T) * T + 0.5))
        specs.append((kc - N // 2, N, N))
        srcs.append([s])
    wins, _, _ = layout(specs, [n_prop] * n_win)
    nA, nE, wA, wE = noise_and_weights(wins, T, rng)
    log_u = log_uniforms(n_win * n_prop, rng)
    wl = Workload("posterior: 16 windows N=128-256, 10k proposals each, T=2 yr", T, wins,
                  nA, nE, wA, wE, srcs, np.zeros((n_win * n_prop, 8)), None, log_u,
                  {"seed": seed, "snr": snr, "proposal_seed": seed + 1000})
    return wl


def band_windows(seed=SEED_BASE + 3, n_win=512, T=YEAR, cand_range=(2000, 20000),
                 f_lo=0.3e-3, f_hi=20e-3, scale_counts=1.0):
    """512 windows log-spaced over 0.3-20 mHz at T = 1 yr with N by band
    (32 / 64 / 128 / 256 / 512 / 1024), 1-4 sources per window (f0 uniform in
    the window, fdot from Eq. 8 with Mc ~ U[0.2, 1] M_sun, A log-uniform in
    [1e-23, 1e-21]) and U{2000..20000} candidates per window around a random
    source of the window."""
    rng = np.random.default_rng(seed)
    centers = np.exp(np.linspace(np.log(f_lo), np.log(f_hi), n_win))
    specs, srcs, counts = [], [], []
    for fc in centers:
        N = n_for_band(fc, T, 1.0)
        N = min(max(N, 32), 1024)
        kc = int(round(fc * T))
        k0 = kc - N // 2
        ns = int(rng.integers(1, 5))
        ss = []
        for _ in range(ns):
            f0 = (k0 + N * 0.25 + rng.uniform(0, 0.5 * N)) / T
            fdot = float(chirp_fdot(f0, rng.uniform(0.2, 1.0)))
            f0 = f0 - 0.5 * fdot * T     # keep the mid-observation frequency inside
            A = float(np.exp(rng.uniform(np.log(1e-23), np.log(1e-21))))
            ss.append(source(f0, fdot, A, rng))
        srcs.append(ss)
        specs.append((k0, N, N))
        counts.append(max(1, int(rng.integers(cand_range[0], cand_range[1] + 1) * scale_counts)))
    wins, _, ntot = layout(specs, counts)
    nA, nE, wA, wE = noise_and_weights(wins, T, rng)
    th = np.empty((ntot, 8))
    for w, (k0, W, N, doff, coff, nc) in enumerate(wins):
        s = srcs[w][int(rng.integers(0, len(srcs[w])))]
        half = np.array([5.0 / T, 0.5 * abs(s[1]) + 1e-20, 0.2, 0.2, 0.5 * s[4], 0.3, 0.3, 0.3])
        th[coff:coff + nc] = uniform_box(s, half, nc, rng)
    th[:, 2] = np.clip(th[:, 2], -np.pi / 2, np.pi / 2)
    return Workload("band: 512 windows 0.3-20 mHz, N=32..1024, 2k-20k candidates, T=1 yr", T, wins,
                    nA, nE, wA, wE, srcs, th, None, log_uniforms(ntot, rng), {"seed": seed})


def population_windows(seed=SEED_BASE + 4, n_win=64, pop=4096, T=2 * YEAR, N=256):
    """64 windows of N = 256 at T = 2 yr, f0 log-uniform in [2, 6.5] mHz, two
    sources per window 3-10 bins apart, a population of 4,096 per window
    uniform in a box spanning both sources."""
    rng = np.random.default_rng(seed)
    specs, srcs = [], []
    for _ in range(n_win):
        f0 = float(np.exp(rng.uniform(np.log(2e-3), np.log(6.5e-3))))
        fd = float(chirp_fdot(f0, rng.uniform(0.2, 1.0)))
        df = rng.uniform(3, 10) / T
        s1 = source(f0, fd, float(np.exp(rng.uniform(np.log(3e-23), np.log(1e-21)))), rng)
        s2 = source(f0 + df, float(chirp_fdot(f0 + df, rng.uniform(0.2, 1.0))),
                    float(np.exp(rng.uniform(np.log(3e-23), np.log(1e-21)))), rng)
        kc = int(math.floor((f0 + 0.5 * df + 0.5 * fd * T) * T + 0.5))
        specs.append((kc - N // 2, N, N))
        srcs.append([s1, s2])
    wins, _, ntot = layout(specs, [pop] * n_win)
    nA, nE, wA, wE = noise_and_weights(wins, T, rng)
    th = np.empty((ntot, 8))
    for w, (k0, W, Nw, doff, coff, nc) in enumerate(wins):
        s1, s2 = srcs[w]
        lo = np.array([min(s1[0], s2[0]) - 3 / T, 0.0, -np.pi / 2, -np.pi, 1e-23, 0.0, 0.0, 0.0])
        hi = np.array([max(s1[0], s2[0]) + 3 / T, 2 * max(s1[1], s2[1]), np.pi / 2, np.pi, 1e-21,
                       np.pi, np.pi, 2 * np.pi])
        th[coff:coff + nc] = lo + (hi - lo) * rng.uniform(0, 1, (nc, 8))
    return Workload("population: 64 windows N=256, 2 sources each, 4096 per window, T=2 yr", T,
                    wins, nA, nE, wA, wE, srcs, th, None, log_uniforms(ntot, rng), {"seed": seed})
