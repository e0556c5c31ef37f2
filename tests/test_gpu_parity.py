"""Parity of the CUDA path (through the C-ABI) with the FP64 oracle.

Bars: the plain-double path matches the oracle to 1e-10 relative (templates
norm-wise; logL, <d|h>, <h|h> per candidate); the mixed path to
|dlogL| <= 1e-3 at SNR ~ 50; chain indices bit-exact; the double gradient
to 1e-9 of the gradient norm (natural parameter units).
"""
import math
import os

import numpy as np
import pytest
import torch

from oracle import gb as ogb
from oracle import mh as omh
from paper_2307_03763_gb300 import workloads as wk
from tests import _data

pytestmark = pytest.mark.gpu

YEAR = wk.YEAR
T2 = 2 * YEAR
DEV = "cuda:0"


@pytest.fixture(scope="session")
def api():
    from paper_2307_03763_gb300 import api, build
    build.build()
    return api


@pytest.fixture(scope="session")
def ctx(api):
    return api.Context(T2)


@pytest.fixture(scope="session")
def ctx1(api):
    return api.Context(YEAR)


def _cuda(x, dtype):
    return torch.as_tensor(np.ascontiguousarray(x)).to(device=DEV, dtype=dtype)


def _thetas(rng, n, f0, T, fd_scale=1.0):
    out = np.stack([wk.source(f0 * (1 + 0.01 * rng.uniform(-1, 1)), 0.0, 1e-22, rng) for _ in range(n)])
    out[:, 1] = fd_scale * wk.chirp_fdot(out[:, 0], rng.uniform(0.2, 1.0, n))
    out[:, 4] = np.exp(rng.uniform(np.log(1e-23), np.log(1e-21), n))
    return out


# --------------------------------------------------------------------------
# templates
# --------------------------------------------------------------------------

# the last two reach the J = 10 and direct link-transfer tiers (f/f* = 1.6, 2.6)
BANDS = [(32, 0.8e-3), (64, 2.5e-3), (128, 5e-3), (256, 9e-3), (512, 14e-3), (1024, 19e-3), (1024, 30e-3),
         (1024, 50e-3)]


@pytest.mark.parametrize("N,f0", BANDS)
def test_waveform_fp64_matches_oracle(ctx1, N, f0):
    rng = np.random.default_rng(100 + N)
    th = _thetas(rng, 37, f0, YEAR)
    hA, hE, q = ctx1.waveform(_cuda(th, torch.float64), N, "fp64")
    qo, oA, oE = ogb.template(torch.tensor(th), N, YEAR)
    assert torch.equal(q.cpu(), qo)
    for g, o in ((hA, oA), (hE, oE)):
        g = g.cpu()
        err = (g - o).abs().amax(1) / o.abs().amax(1)
        assert err.max() < 1e-10, err.max()


@pytest.mark.parametrize("N,f0", BANDS)
def test_waveform_mixed_close_to_oracle(ctx1, N, f0):
    rng = np.random.default_rng(200 + N)
    th = _thetas(rng, 37, f0, YEAR)
    hA, hE, q = ctx1.waveform(_cuda(th, torch.float64), N, "mixed")
    qo, oA, oE = ogb.template(torch.tensor(th), N, YEAR)
    assert torch.equal(q.cpu(), qo)
    for g, o in ((hA, oA), (hE, oE)):
        err = (g.cpu() - o).abs().amax(1) / o.abs().amax(1)
        assert err.max() < 2e-6, err.max()


def test_waveform_empty_batch(ctx):
    hA, hE, q = ctx.waveform(torch.zeros((0, 8), dtype=torch.float64, device=DEV), 64)
    assert hA.shape == (0, 64) and q.shape == (0,)


# --------------------------------------------------------------------------
# log-likelihood
# --------------------------------------------------------------------------

def _run_both(ctx, wins, dA, dE, wA, wE, th, T, prec):
    args = (_cuda(dA, torch.complex128), _cuda(dE, torch.complex128), _cuda(wA, torch.float64),
            _cuda(wE, torch.float64), _cuda(th, torch.float64))
    g = [x.cpu() for x in ctx.loglik(wins, *args, prec=prec)]
    o = ogb.loglik(wins, dA, dE, wA, wE, th, T)
    return g, o


def _assert_close_fp64(g, o, rows=None):
    gl, gdh, ghh = g
    ol, odh, ohh = o
    if rows is not None:
        gl, gdh, ghh, ol, odh, ohh = (x[rows] for x in (gl, gdh, ghh, ol, odh, ohh))
    scale = max(1.0, float(ohh.abs().max()))
    assert ((gl - ol).abs() <= 1e-10 * torch.clamp(ol.abs(), min=1.0)).all(), (gl - ol).abs().max()
    assert ((gdh - odh).abs() <= 1e-10 * scale).all(), (gdh - odh).abs().max()
    assert ((ghh - ohh).abs() <= 1e-10 * scale).all(), (ghh - ohh).abs().max()


def test_loglik_fp64_tiny_window_full(ctx):
    # one window of N = 128 at 1.5 mHz, 1,000 candidates (every output checked)
    wl = wk.tiny_window()
    dA, dE = _data.inject(wl)
    g, o = _run_both(ctx, wl.windows, dA, dE, wl.w_A, wl.w_E, wl.theta, wl.T, "fp64")
    _assert_close_fp64(g, o)
    assert float(g[2].max()) > 100.0       # the injected source is seen (SNR^2 scale)


def test_loglik_fp64_ragged_windows(ctx):
    # several windows in one launch: different N, W != N, templates partly or
    # wholly outside, an empty window, W = 0, ragged candidate counts
    rng = np.random.default_rng(7)
    T = T2
    specs = []
    th_all, counts = [], []
    for (N, f0, W, shift, nc) in [(32, 0.6e-3, 32, 0, 1), (64, 1.1e-3, 80, -20, 33), (128, 2.0e-3, 128, 45, 129),
                                  (256, 3.9e-3, 200, 0, 257), (128, 2.4e-3, 128, 0, 0), (64, 1.5e-3, 0, 0, 5),
                                  (512, 4.5e-3, 512, -300, 40), (1024, 5.0e-3, 1024, 0, 19),
                                  (128, 1.7e-3, 128, 10 ** 6, 7)]:
        src = wk.source(f0, float(wk.chirp_fdot(f0, 0.6)), 3e-22, rng)
        kc = int(math.floor((src[0] + 0.5 * src[1] * T) * T + 0.5))
        specs.append((kc - W // 2 + shift, W, N))
        half = np.array([3.0 / T, abs(src[1]), 0.3, 0.3, 0.5 * src[4], 0.3, 0.3, 0.3])
        th_all.append(wk.uniform_box(src, half, nc, rng))
        counts.append(nc)
    wins, nb, nt = wk.layout(specs, counts)
    nA, nE, wA, wE = wk.noise_and_weights(wins, T, rng)
    th = np.concatenate(th_all)
    srcs = [[th_all[i][0]] if counts[i] else [] for i in range(len(specs))]
    wl = wk.Workload("ragged", T, wins, nA, nE, wA, wE, srcs, th)
    dA, dE = _data.inject(wl)
    g, o = _run_both(ctx, wins, dA, dE, wA, wE, th, T, "fp64")
    _assert_close_fp64(g, o)


def test_loglik_mixed_tolerance_at_snr50(ctx):
    wl = wk.tiny_window(seed=wk.SEED_BASE + 11)
    src = wl.sources[0][0].copy()
    rho1 = _data.unit_snr(src, wl.windows[0], wl.w_A, wl.w_E, wl.T)
    scale = 50.0 / rho1
    src[4] *= scale
    wl.theta[:, 4] *= scale
    dA, dE = _data.inject(wl, [[src]])
    g, o = _run_both(ctx, wl.windows, dA, dE, wl.w_A, wl.w_E, wl.theta, wl.T, "mixed")
    dl = (g[0] - o[0]).abs()
    assert float(o[2].max()) > 1000.0
    assert float(dl.max()) <= 1e-3, float(dl.max())


def test_loglik_mixed_multiband(ctx1):
    # every N / band of the 0.3-20 mHz workload, a few windows each
    wl = wk.band_windows(n_win=12, cand_range=(50, 90))
    dA, dE = _data.inject(wl)
    g, o = _run_both(ctx1, wl.windows, dA, dE, wl.w_A, wl.w_E, wl.theta, wl.T, "mixed")
    rel = (g[0] - o[0]).abs() / torch.clamp(o[2].abs(), min=1.0)
    assert float(rel.max()) < 1e-5, float(rel.max())
    gf, of = _run_both(ctx1, wl.windows, dA, dE, wl.w_A, wl.w_E, wl.theta, wl.T, "fp64")
    _assert_close_fp64(gf, of)


def _fixed_point_problem(f0, fd_scale, seed):
    # one window of N = 64 and one of N = 256, each with an injected source at
    # f0 and 24 candidates in a small box around it (carrier bins in the
    # window), T = 1 yr
    rng = np.random.default_rng(seed)
    T = YEAR
    specs, th, srcs = [], [], []
    for N in (64, 256):
        src = wk.source(f0, fd_scale * float(wk.chirp_fdot(f0, 0.5)), 2e-21, rng)
        if f0 > 60e-3:
            src[2], src[3] = 0.1, 0.2          # |f0 Kc| near 31 cycles: the box straddles the bound
        half = np.array([3.0 / T, 1e-3 * abs(src[1]), 0.3, 0.3, 0.1 * src[4], 0.1, 0.1, 0.1])
        t = wk.uniform_box(src, half, 24, rng)
        kc = int(math.floor((src[0] + 0.5 * src[1] * T) * T + 0.5))
        specs.append((kc - N // 2, N, N))
        th.append(t)
        srcs.append([src])
    wins, _, _ = wk.layout(specs, [24, 24])
    nA, nE, wA, wE = wk.noise_and_weights(wins, T, rng)
    return wk.Workload("fixed-point ranges", T, wins, nA, nE, wA, wE, srcs, np.concatenate(th))


@pytest.mark.parametrize("f0,fd_scale", [(30e-3, 0.1), (64e-3, 0.01), (70e-3, 0.01), (5e-3, 4000.0)])
def test_mixed_fixed_point_phase_ranges(ctx1, f0, fd_scale):
    # the paired slow part takes the carrier phase in fixed point while
    # |f0 K| < 31 cycles (K = -(AU/c) cos(beta) (cos lambda, sin lambda)) and
    # in double-word floats beyond (f0 above ~62 mHz; 64 and 70 mHz put
    # candidates on both sides in one launch); the last case chirps by
    # thousands of cycles over T (fdot T^2/2 reduced modulo 2^20 in fixed
    # point).  Likelihood and gradient against the oracle at the multiband bars.
    wl = _fixed_point_problem(f0, fd_scale, int(f0 * 1e5) + int(fd_scale))
    th = wl.theta
    kpart = f0 * 149597870700.0 / 299792458.0 * np.cos(th[:, 2])
    wide = (np.abs(kpart * np.cos(th[:, 3])) >= 31.0) | (np.abs(kpart * np.sin(th[:, 3])) >= 31.0)
    if f0 >= 64e-3:
        assert wide.any() and not wide.all()              # both forms in one launch
    else:
        assert not wide.any()
    if fd_scale > 1.0:
        assert float(np.max(0.5 * np.abs(th[:, 1]) * wl.T ** 2)) > 1000.0
    dA, dE = _data.inject(wl)
    g, o = _run_both(ctx1, wl.windows, dA, dE, wl.w_A, wl.w_E, th, wl.T, "mixed")
    rel = (g[0] - o[0]).abs() / torch.clamp(o[2].abs(), min=1.0)
    assert float(rel.max()) < 1e-5, float(rel.max())
    assert float(o[2].max()) > 1.0                       # the injected source is seen
    args = (_cuda(dA, torch.complex128), _cuda(dE, torch.complex128), _cuda(wl.w_A, torch.float64),
            _cuda(wl.w_E, torch.float64), _cuda(th, torch.float64))
    lg, gg = (x.cpu() for x in ctx1.loglik_grad(wl.windows, *args, prec="mixed"))
    lo, go = ogb.loglik_grad(wl.windows, dA, dE, wl.w_A, wl.w_E, th, wl.T)
    worst = 0.0
    for b in range(th.shape[0]):
        s = torch.tensor([1 / wl.T, 1 / wl.T ** 2, 1, 1, th[b, 4], 1, 1, 1], dtype=torch.float64)
        gn, on = gg[b] * s, go[b] * s
        worst = max(worst, float((gn - on).abs().max()) / float(on.abs().sum()))
    assert worst <= 1e-4, worst


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_loglik_phase_is_dh_at_a_quarter_turn(ctx1, prec):
    # gb_loglik_phase: dh_im(theta) = <d|h> at phi0 + pi/2 (oracle), every N
    # of the band workload; logL, dh, hh are those of gb_loglik
    wl = wk.band_windows(seed=wk.SEED_BASE + 21, n_win=12, cand_range=(40, 70))
    dA, dE = _data.inject(wl)
    args = (_cuda(dA, torch.complex128), _cuda(dE, torch.complex128), _cuda(wl.w_A, torch.float64),
            _cuda(wl.w_E, torch.float64), _cuda(wl.theta, torch.float64))
    lp, dp, dip, hp = (x.cpu() for x in ctx1.loglik_phase(wl.windows, *args, prec=prec))
    lg, dg, hg = (x.cpu() for x in ctx1.loglik(wl.windows, *args, prec=prec))
    tq = wl.theta.copy()
    tq[:, 7] += np.pi / 2
    _, oq, ohh = ogb.loglik(wl.windows, dA, dE, wl.w_A, wl.w_E, tq, wl.T)
    if prec == "fp64":
        assert torch.equal(lp, lg) and torch.equal(dp, dg) and torch.equal(hp, hg)
        scale = max(1.0, float(ohh.abs().max()))
        assert float((dip - oq).abs().max()) <= 1e-10 * scale
    else:
        assert float((lp - lg).abs().max()) <= 1e-9 * max(1.0, float(hg.abs().max()))
        rel = (dip - oq).abs() / torch.clamp(ohh.abs(), min=1.0)
        assert float(rel.max()) < 1e-5, float(rel.max())


def test_loglik_phase_mixed_at_snr50(ctx):
    # the imaginary part meets the mixed path's bar at SNR ~ 50
    wl = wk.tiny_window(seed=wk.SEED_BASE + 11)
    src = wl.sources[0][0].copy()
    scale = 50.0 / _data.unit_snr(src, wl.windows[0], wl.w_A, wl.w_E, wl.T)
    src[4] *= scale
    wl.theta[:, 4] *= scale
    dA, dE = _data.inject(wl, [[src]])
    args = (_cuda(dA, torch.complex128), _cuda(dE, torch.complex128), _cuda(wl.w_A, torch.float64),
            _cuda(wl.w_E, torch.float64), _cuda(wl.theta, torch.float64))
    _, _, dip, _ = (x.cpu() for x in ctx.loglik_phase(wl.windows, *args, prec="mixed"))
    tq = wl.theta.copy()
    tq[:, 7] += np.pi / 2
    _, oq, _ = ogb.loglik(wl.windows, dA, dE, wl.w_A, wl.w_E, tq, wl.T)
    assert float(oq.abs().max()) > 1000.0
    assert float((dip - oq).abs().max()) <= 1e-3


def mixed_bound(l, dh, hh, eps, cf=1e-6):
    """Per-row bound of |logL_mixed - logL_fp64| from the mixed outputs (the
    model gb_mh_certified settles decisions with): eps |h| |d - h| +
    eps^2 |h|^2 / 2 + cf |h| (|d| + |h|) + 1e-12 (|logL| + |d|^2 + |h|^2), with
    <d|d> = 2 (dh - hh/2 - logL) and |d - h| <= (-2 logL)^1/2 + eps |h|."""
    dd = (2.0 * (dh - 0.5 * hh - l)).abs()
    h2 = hh.clamp(min=0.0)
    nh = h2.sqrt()
    nr = (-2.0 * l).clamp(min=0.0).sqrt() + eps * nh
    return eps * nh * nr + 0.5 * eps * eps * h2 + cf * nh * (dd.sqrt() + nh) + 1e-12 * (l.abs() + dd + h2)


def test_loglik_posterior_workload_sampled(ctx, api):
    # the 16-window, 10,000-proposal workload at full size in one launch, in
    # both precisions.  Every row: the mixed value within half the bound of
    # the certified chains (eps = api.MIXED_EPS) of the FP64 path's; the FP64
    # path against the oracle on sampled rows (first, last and 40 random rows
    # per window) at 1e-10, and the mixed path there against the oracle too
    wl = wk.posterior_windows()
    rng = np.random.default_rng(5)
    srcs = []
    th = np.empty((wl.n_cand, 8))
    for w, (k0, W, N, doff, coff, nc) in enumerate(wl.windows):
        s = wl.sources[w][0].copy()
        s[4] = wl.meta["snr"][w] / _data.unit_snr(s, wl.windows[w], wl.w_A, wl.w_E, wl.T)
        srcs.append([s])
        sig = _data.fisher_sigma(s, wl.windows[w], wl.w_A, wl.w_E, wl.T)
        th[coff:coff + nc], _ = wk.gaussian_proposals(s, 10 * sig, nc, rng)
    dA, dE = _data.inject(wl, srcs)
    args = (_cuda(dA, torch.complex128), _cuda(dE, torch.complex128), _cuda(wl.w_A, torch.float64),
            _cuda(wl.w_E, torch.float64), _cuda(th, torch.float64))
    g64 = [x.cpu() for x in ctx.loglik(wl.windows, *args, prec="fp64")]
    gmx = [x.cpu() for x in ctx.loglik(wl.windows, *args, prec="mixed")]
    # every row against the FP64 GPU path
    dl = (gmx[0] - g64[0]).abs()
    bound = mixed_bound(gmx[0], gmx[1], gmx[2], api.MIXED_EPS)
    assert bool(torch.isfinite(gmx[0]).all())
    assert bool((dl <= 0.5 * bound).all()), float((dl / bound).max())
    # per SNR band of the proposal (<h|h>^1/2): max |dlogL| <= 0.5 eps SNR (SNR_d + SNR)
    snr = g64[2].sqrt()
    snr_d = (2.0 * (g64[1] - 0.5 * g64[2] - g64[0])).abs().sqrt()
    for lo, hi in [(0, 20), (20, 50), (50, 100), (100, 200), (200, 1e9)]:
        m = (snr >= lo) & (snr < hi)
        if bool(m.any()):
            assert float(dl[m].max()) <= 0.5 * api.MIXED_EPS * float((snr[m] * (snr_d[m] + snr[m])).max())
    rows = []
    for (k0, W, N, doff, coff, nc) in wl.windows:
        rows += [coff, coff + nc - 1] + list(coff + rng.choice(nc, 40, replace=False))
    rows = np.array(sorted(set(rows)))
    sub_wins, sub_th = [], []
    for (k0, W, N, doff, coff, nc) in wl.windows:
        sel = rows[(rows >= coff) & (rows < coff + nc)]
        sub_wins.append((k0, W, N, doff, len(sub_th), len(sel)))
        sub_th += list(th[sel])
    o = ogb.loglik(sub_wins, dA, dE, wl.w_A, wl.w_E, np.array(sub_th), wl.T)
    idx = torch.tensor(rows)
    _assert_close_fp64([x[idx] for x in g64], o)
    assert bool(((gmx[0][idx] - o[0]).abs() <= 0.5 * bound[idx] + 1e-10 * o[0].abs().clamp(min=1.0)).all())


def test_loglik_outputs_optional(ctx):
    wl = wk.tiny_window(n_cand=40)
    dA, dE = _data.inject(wl)
    args = (_cuda(dA, torch.complex128), _cuda(dE, torch.complex128), _cuda(wl.w_A, torch.float64),
            _cuda(wl.w_E, torch.float64), _cuda(wl.theta, torch.float64))
    logL = torch.zeros(40, dtype=torch.float64, device=DEV)
    for prec in ("fp64", "mixed"):
        l1, _, _ = ctx.loglik(wl.windows, *args, prec=prec)
        ctx.loglik(wl.windows, *args, prec=prec, out=(logL, None, None))
        assert torch.equal(l1, logL)


def test_nonfinite_parameter_gives_nan_and_status(ctx, api):
    wl = wk.tiny_window(n_cand=8)
    th = wl.theta.copy()
    th[3, 2] = np.nan
    th[5, 0] = np.inf
    args = (_cuda(wl.noise_A, torch.complex128), _cuda(wl.noise_E, torch.complex128),
            _cuda(wl.w_A, torch.float64), _cuda(wl.w_E, torch.float64), _cuda(th, torch.float64))
    for prec in ("fp64", "mixed"):
        l, _, _ = ctx.loglik(wl.windows, *args, prec=prec)
        l = l.cpu()
        assert math.isnan(l[3]) and math.isnan(l[5]) and torch.isfinite(l[[0, 1, 2, 4, 6, 7]]).all()
        with pytest.raises(api.GBError):
            ctx.check()
        ctx.check()     # cleared


def test_argument_errors_raise(ctx, api):
    wl = wk.tiny_window(n_cand=8)
    args = [_cuda(wl.noise_A, torch.complex128), _cuda(wl.noise_E, torch.complex128),
            _cuda(wl.w_A, torch.float64), _cuda(wl.w_E, torch.float64), _cuda(wl.theta, torch.float64)]
    k0, W, N, doff, coff, nc = wl.windows[0]
    for bad in ([(k0, W, 100, doff, coff, nc)], [(k0, W, 2048, doff, coff, nc)],
                [(k0, W + 1, N, doff, coff, nc)], [(k0, W, N, doff, coff + 1, nc)],
                [(k0, -1, N, doff, coff, nc)]):
        with pytest.raises(api.GBError):
            ctx.loglik(bad, *args)
    with pytest.raises(api.GBError):
        ctx.waveform(args[4], 48)


# --------------------------------------------------------------------------
# Metropolis-Hastings chains
# --------------------------------------------------------------------------

def _mh_both(ctx, L, G, U, T, literal):
    chain, acc = ctx.mh_independence(_cuda(L, torch.float64), _cuda(G, torch.float64), _cuda(U, torch.float64),
                                     _cuda(T, torch.float64), literal=literal)
    oc, oa = omh.mh_independence_batch(L, G, U, T, literal)
    return chain.cpu().numpy(), acc.cpu().numpy(), np.array(oc), np.array(oa)


@pytest.mark.parametrize("literal", [False, True])
def test_mh_matches_oracle_full_size(ctx, literal):
    rng = np.random.default_rng(11)
    nch, n = 16, 10000
    L = rng.normal(-50, 4, (nch, n))
    G = rng.normal(0, 2, (nch, n))
    U = np.log(rng.uniform(0, 1, (nch, n)))
    T = np.array([1.0, 2.0, 3.0, 5.0, 10.0, 15.0] * 3)[:nch]
    c, a, oc, oa = _mh_both(ctx, L, G, U, T, literal)
    assert np.array_equal(c, oc)
    assert np.array_equal(a, oa)


@pytest.mark.parametrize("T,literal", [(1.0, False), (3.0, False), (3.0, True)])
def test_mh_near_ties_match_oracle(ctx, T, literal):
    # log u placed exactly on, or one ulp below, the acceptance boundary
    # Delta of the current state, so that the decision needs the full double
    # expression; the oracle run on the same inputs fixes the expected chain
    rng = np.random.default_rng(21)
    n = 4000
    L = rng.normal(-40.0, 5.0, n)
    G = rng.normal(0.0, 1.0, n)
    w = (L - G) if literal else (L / T - G)
    U = np.log(rng.uniform(0, 1, n))
    c = 0
    for i in range(1, n):
        d = (w[i] - w[c]) / T if literal else w[i] - w[c]
        if d < 0 and rng.uniform() < 0.5:
            U[i] = d if rng.uniform() < 0.5 else np.nextafter(d, -np.inf)
        if U[i] < min(0.0, d):
            c = i
    cg, ag, co, ao = _mh_both(ctx, L[None], G[None], U[None], np.array([T]), literal)
    assert np.array_equal(cg, co) and np.array_equal(ag, ao)


def test_mh_golden_and_edge_cases(ctx):
    path = os.path.join(os.path.dirname(__file__), "golden", "mh_alg4_worked.txt")
    g = {}
    for line in open(path):
        if "=" in line and not line.startswith("#"):
            k, v = line.strip().split("=")
            g[k] = [float(x) for x in v.split(",")]
    c, a, _, _ = _mh_both(ctx, np.array([g["logL"]]), np.array([g["log_g"]]), np.array([g["log_u"]]),
                          np.array(g["temperature"]), False)
    assert c[0].tolist() == [int(x) for x in g["chain"]] and a[0] == int(g["n_accept"][0])
    # ragged lengths not multiple of the prefetch depth, n = 1, -inf entries
    for n in (1, 2, 9, 17):
        rng = np.random.default_rng(n)
        L = rng.normal(0, 1, (3, n))
        L[:, n // 2] = -np.inf
        c, a, oc, oa = _mh_both(ctx, L, rng.normal(0, 1, (3, n)), np.log(rng.uniform(0, 1, (3, n))),
                                np.ones(3), False)
        assert np.array_equal(c, oc) and np.array_equal(a, oa)


def _mh_adversarial_rows(rng, n):
    """Rows that reach every path of the chunked scan: sorted weights (more
    records per chunk than are summarised), special values, weights of 1e20
    where the first threshold guess is many doubles off, tiny |log u|."""
    rows = []
    L = np.sort(rng.normal(0, 50, n))
    rows.append((L, np.zeros(n), np.log(rng.uniform(size=n))))
    L, G, U = rng.normal(0, 3, n), rng.normal(0, 1, n), np.log(rng.uniform(size=n))
    for a in (L, G, U):
        m = rng.uniform(size=n) < 0.02
        a[m] = rng.choice([np.inf, -np.inf, np.nan, 0.0, -0.0], m.sum())
    rows.append((L, G, U))
    rows.append((1e20 + rng.integers(-4, 4, n) * 16384.0, -1e20 + rng.integers(-4, 4, n) * 16384.0,
                 np.log(rng.uniform(size=n))))
    rows.append((np.round(rng.normal(0, 3, n)), np.zeros(n), -rng.uniform(0, 1e-18, n)))
    rows.append((rng.normal(-50, 4, n), rng.normal(0, 2, n), np.log(rng.uniform(size=n))))
    return [np.stack(x) for x in zip(*rows)]


@pytest.mark.parametrize("literal", [False, True])
def test_mh_chunked_scan_adversarial(ctx, literal):
    # every chain length around the chunk size, and one long enough that the
    # chunk summaries are combined in several batches; temperatures that keep
    # the threshold form (positive, finite) and ones that do not (literal form)
    rng = np.random.default_rng(31 + literal)
    temps = np.array([1.0, 0.7, 3.0, -2.0, np.inf, np.nan, 1e-300, 1e300])
    for n in (2, 31, 511, 512, 513, 514, 1025, 40001):
        L, G, U = _mh_adversarial_rows(rng, n)
        rows = len(L)
        for T in temps:
            c, a, oc, oa = _mh_both(ctx, L, G, U, np.full(rows, T), literal)
            assert np.array_equal(c, oc), (n, T, np.argwhere(c != oc)[:5])
            assert np.array_equal(a, oa), (n, T)


# --------------------------------------------------------------------------
# gradient
# --------------------------------------------------------------------------

@pytest.mark.parametrize("which", ["tiny", "band"])
def test_grad_mixed_matches_oracle(ctx, ctx1, which):
    # mixed-precision adjoint against the oracle's gradient, per candidate, in
    # natural parameter units, relative to the gradient norm
    if which == "tiny":
        wl, c = wk.tiny_window(n_cand=40), ctx
    else:
        wl, c = wk.band_windows(n_win=10, cand_range=(6, 9)), ctx1
    dA, dE = _data.inject(wl)
    th = wl.theta.copy()
    args = (_cuda(dA, torch.complex128), _cuda(dE, torch.complex128), _cuda(wl.w_A, torch.float64),
            _cuda(wl.w_E, torch.float64), _cuda(th, torch.float64))
    lg, gg = (x.cpu() for x in c.loglik_grad(wl.windows, *args, prec="mixed"))
    lo, go = ogb.loglik_grad(wl.windows, dA, dE, wl.w_A, wl.w_E, th, wl.T)
    worst = 0.0
    for b in range(th.shape[0]):
        s = torch.tensor([1 / wl.T, 1 / wl.T ** 2, 1, 1, th[b, 4], 1, 1, 1], dtype=torch.float64)
        gn, on = gg[b] * s, go[b] * s
        worst = max(worst, float((gn - on).abs().max()) / float(on.abs().sum()))
    assert worst <= 1e-4, worst
    # the likelihood kernel's logL: the same float arithmetic up to the order of
    # the transform's operations (the two kernels factor the DFT differently)
    lm, _, _ = c.loglik(wl.windows, *args, prec="mixed")
    assert torch.allclose(lg, lm.cpu(), rtol=0, atol=1e-6 * float(lo.abs().max()))


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_autotune_keeps_results(api, prec):
    # the tuner changes launch shapes only: outputs stay bit-identical
    wl = wk.band_windows(n_win=16, cand_range=(200, 600))
    c = api.Context(wl.T)
    args = (_cuda(wl.noise_A, torch.complex128), _cuda(wl.noise_E, torch.complex128), _cuda(wl.w_A, torch.float64),
            _cuda(wl.w_E, torch.float64), _cuda(wl.theta, torch.float64))
    before = [x.clone() for x in c.loglik(wl.windows, *args, prec=prec)]
    t = c.autotune(wl.windows, *args, prec=prec, reps=2)
    after = c.loglik(wl.windows, *args, prec=prec)
    for x, y in zip(before, after):
        assert torch.equal(x, y)
    assert t["ms"] <= t["ms_default"] + 1e-9
    if prec == "mixed":
        assert t["item"] in (0, 2, 4, 8, 16, 32) and t["blocks_per_sm"] in (0, 1, 2, 3)
    else:
        assert t["tile"] in (0, 16, 32, 64, 128)


@pytest.mark.parametrize("N", [32, 64, 128])
def test_grad_fp64_matches_oracle(ctx, N):
    wl = wk.tiny_window(n_cand=24, N=N)
    dA, dE = _data.inject(wl)
    th = wl.theta.copy()
    args = (_cuda(dA, torch.complex128), _cuda(dE, torch.complex128), _cuda(wl.w_A, torch.float64),
            _cuda(wl.w_E, torch.float64), _cuda(th, torch.float64))
    lg, gg = (x.cpu() for x in ctx.loglik_grad(wl.windows, *args, prec="fp64"))
    lo, go = ogb.loglik_grad(wl.windows, dA, dE, wl.w_A, wl.w_E, th, wl.T)
    s = torch.tensor([1 / wl.T, 1 / wl.T ** 2, 1, 1, 1, 1, 1, 1], dtype=torch.float64)
    for b in range(th.shape[0]):
        sb = s.clone()
        sb[4] = th[b, 4]
        gn, on = gg[b] * sb, go[b] * sb
        assert float((gn - on).abs().max()) <= 1e-9 * float(on.abs().sum()), (b, gn, on)
    assert ((lg - lo).abs() <= 1e-10 * lo.abs()).all()


@pytest.mark.parametrize("N,f0", [(64, 0.9e-3), (128, 1.5e-3), (256, 4.5e-3), (1024, 1.6e-2)])
def test_grad_fp64_matches_central_differences(ctx, N, f0):
    # the adjoint FP64 gradient against central differences of the FP64
    # likelihood itself, steps of 1e-6 of each parameter's natural scale
    # (1/T, 1/T^2, rad, A), at candidates whose carrier bin q stays fixed
    # under the steps; bar 1e-6 of the gradient's norm (natural units)
    rng = np.random.default_rng(N)
    T = T2
    src = wk.source(f0, float(wk.chirp_fdot(f0, 0.5)), 5e-22, rng)
    kc = int(math.floor((src[0] + 0.5 * src[1] * T) * T + 0.5))
    wins, _, _ = wk.layout([(kc - N // 2, N, N)], [8])
    nA, nE, wA, wE = wk.noise_and_weights(wins, T, rng)
    half = np.array([3.0 / T, abs(src[1]), 0.1, 0.1, 0.1 * src[4], 0.1, 0.1, 0.1])
    th = wk.uniform_box(src, half, 64, rng)
    frac = (th[:, 0] * T + 0.5 * th[:, 1] * T * T + 0.5) % 1.0
    th = th[(frac > 1e-3) & (frac < 1 - 1e-3)][:8]          # q fixed under the steps
    wl = wk.Workload("fd", T, wins, nA, nE, wA, wE, [[src]], th)
    dA, dE = _data.inject(wl)
    data = (_cuda(dA, torch.complex128), _cuda(dE, torch.complex128), _cuda(wA, torch.float64),
            _cuda(wE, torch.float64))
    nb = th.shape[0]
    _, gg = (x.cpu() for x in ctx.loglik_grad([(wins[0][0], N, N, 0, 0, nb)], *data, _cuda(th, torch.float64),
                                              prec="fp64"))
    scale = np.stack([np.array([1 / T, 1 / T ** 2, 1, 1, th[b, 4], 1, 1, 1]) for b in range(nb)])
    pts, h = [], np.empty((8, nb))
    for i in range(8):
        tp, tm = th.copy(), th.copy()
        tp[:, i] += 1e-6 * scale[:, i]
        tm[:, i] -= 1e-6 * scale[:, i]
        pts += [tp, tm]
        # the step actually taken, from the doubles.  f0 enters the phase
        # through delta = fl(f0 T) - q (all but ~1e-5 of d logL/d f0), and
        # f0 T ~ 1e5 is rounded to ~1e-11 cycles, so for f0 the step is the
        # change of the rounded product fl(f0 T) (IEEE products, as the kernel's)
        h[i] = (tp[:, i] - tm[:, i]) / scale[:, i]
        if i == 0:
            h[i] = tp[:, 0] * T - tm[:, 0] * T
    allp = np.concatenate(pts)
    l, _, _ = ctx.loglik([(wins[0][0], N, N, 0, 0, allp.shape[0])], *data, _cuda(allp, torch.float64), prec="fp64")
    l = l.cpu().numpy().reshape(8, 2, nb)
    fd = ((l[:, 0] - l[:, 1]) / h).T                         # d logL / d(theta_i / scale_i)
    adj = gg.numpy() * scale
    for b in range(nb):
        assert np.max(np.abs(adj[b] - fd[b])) <= 1e-6 * np.sum(np.abs(fd[b])), (b, adj[b], fd[b])


def test_autograd_function_uses_the_adjoint(ctx):
    from paper_2307_03763_gb300 import autograd as ag
    wl = wk.tiny_window(n_cand=12)
    dA, dE = _data.inject(wl)
    data = (_cuda(dA, torch.complex128), _cuda(dE, torch.complex128), _cuda(wl.w_A, torch.float64),
            _cuda(wl.w_E, torch.float64))
    th = _cuda(wl.theta, torch.float64).requires_grad_(True)
    for prec in ("fp64", "mixed"):
        l = ag.loglik(ctx, wl.windows, *data, th, prec=prec)
        wts = torch.linspace(0.5, 2.0, 12, dtype=torch.float64, device=DEV)
        (g,) = torch.autograd.grad((l * wts).sum(), th)
        _, gd = ctx.loglik_grad(wl.windows, *data, th.detach(), prec=prec)
        assert torch.allclose(g, gd * wts[:, None], rtol=1e-12, atol=0)


def test_observed_fisher_matches_oracle_fisher(ctx):
    # noise-free data at the truth: -d2 logL = J^T W J exactly
    from paper_2307_03763_gb300 import autograd as ag
    wl = wk.tiny_window(seed=wk.SEED_BASE + 50, n_cand=1)
    src = wl.sources[0][0].copy()
    src[4] *= 50.0 / _data.unit_snr(src, wl.windows[0], wl.w_A, wl.w_E, wl.T)
    hA, hE = _data.template_on_window(src, *wl.windows[0][:3], wl.T)
    data = (_cuda(hA, torch.complex128), _cuda(hE, torch.complex128), _cuda(wl.w_A, torch.float64),
            _cuda(wl.w_E, torch.float64))
    F = ag.observed_fisher(ctx, wl.windows, *data, _cuda(src[None], torch.float64), prec="fp64")[0].cpu().numpy()
    ref = _data.fisher_matrix(src, wl.windows[0], wl.w_A, wl.w_E, wl.T)
    sc = np.array([1 / wl.T, 1 / wl.T ** 2, 1, 1, src[4], 1, 1, 1])
    Fs, Rs = F * np.outer(sc, sc), ref * np.outer(sc, sc)
    d = np.sqrt(np.outer(np.diag(Rs), np.diag(Rs)))
    assert np.abs(Fs - Rs).max() <= 1e-5 * d.max() and (np.abs(Fs - Rs) / d).max() < 1e-4, (Fs, Rs)
    assert np.all(np.linalg.eigvalsh(Fs) > -1e-9 * d.max())


def test_expected_fisher_matches_oracle_fisher(ctx1):
    # F = <d_i h|d_j h> at one source per window, every N of the band workload
    from paper_2307_03763_gb300 import autograd as ag
    wl = wk.band_windows(n_win=10, cand_range=(1, 2))
    src = np.stack([wl.sources[w][0] for w in range(len(wl.windows))])
    for w in range(len(wl.windows)):
        src[w, 4] *= 50.0 / _data.unit_snr(src[w], wl.windows[w], wl.w_A, wl.w_E, wl.T)
    F = ag.expected_fisher(ctx1, wl.windows, _cuda(wl.w_A, torch.float64), _cuda(wl.w_E, torch.float64),
                           _cuda(src, torch.float64)).cpu().numpy()
    assert sorted({w[2] for w in wl.windows}) == [32, 64, 128, 256, 512, 1024]
    for w in range(len(wl.windows)):
        ref = _data.fisher_matrix(src[w], wl.windows[w], wl.w_A, wl.w_E, wl.T)
        sc = np.array([1 / wl.T, 1 / wl.T ** 2, 1, 1, src[w, 4], 1, 1, 1])
        Fs, Rs = F[w] * np.outer(sc, sc), ref * np.outer(sc, sc)
        d = np.sqrt(np.outer(np.diag(Rs), np.diag(Rs)))
        assert np.abs(Fs - Rs).max() <= 1e-5 * d.max() and (np.abs(Fs - Rs) / d).max() < 1e-4, (w, Fs, Rs)


def test_time_budget_stops_persistent_kernels(api):
    # 1 ns: no warp takes an item; a fifth of the launch time: some do.  The
    # rows of the items not taken stay as they were and the check reports it.
    # many small items per warp (one N = 128 window, 200,000 candidates)
    wl = wk.tiny_window(n_cand=200000)
    ctx = api.Context(wl.T)
    data = (_cuda(wl.noise_A, torch.complex128), _cuda(wl.noise_E, torch.complex128), _cuda(wl.w_A, torch.float64),
            _cuda(wl.w_E, torch.float64))
    th = _cuda(wl.theta, torch.float64)
    n = wl.n_cand
    g = torch.empty((n, 8), dtype=torch.float64, device=DEV)
    logL = torch.empty(n, dtype=torch.float64, device=DEV)

    def run(grad):
        if grad:
            ctx.loglik_grad(wl.windows, *data, th, prec="mixed", out=(logL, g))
        else:
            ctx.loglik(wl.windows, *data, th, prec="mixed", out=(logL, None, None))

    for grad in (False, True):
        run(grad)
        ctx.check()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        run(grad)
        b.record()
        torch.cuda.synchronize()
        full_s = a.elapsed_time(b) * 1e-3
        for budget, partial in ((1e-9, False), (0.2 * full_s, True)):
            logL.fill_(float("nan"))
            ctx.set_time_budget(budget)
            run(grad)
            with pytest.raises(api.GBError) as err:
                ctx.check()
            assert err.value.code == api.GB_ETIMEOUT
            left = int(torch.isnan(logL).sum())
            assert (0 < left < n) if partial else (left > 0), (grad, budget, left, n)
        ctx.set_time_budget(0.0)
        logL.fill_(float("nan"))
        run(grad)
        ctx.check()
        assert not bool(torch.isnan(logL).any())
    with pytest.raises(api.GBError):
        ctx.set_time_budget(-1.0)


def test_kernel_events_bracket_the_likelihood_kernels(api):
    # the events set on the context are recorded once, around the likelihood
    # kernels of the next mixed call only: inside the call's own interval,
    # not touched by a later call; one event without the other is refused
    wl = wk.tiny_window(n_cand=20000)
    ctx = api.Context(wl.T)
    data = (_cuda(wl.noise_A, torch.complex128), _cuda(wl.noise_E, torch.complex128), _cuda(wl.w_A, torch.float64),
            _cuda(wl.w_E, torch.float64))
    th = _cuda(wl.theta, torch.float64)
    logL = torch.empty(wl.n_cand, dtype=torch.float64, device=DEV)
    call = lambda: ctx.loglik(wl.windows, *data, th, prec="mixed", out=(logL, None, None))
    call()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    for e in ev:
        e.record()
    with pytest.raises(ValueError):
        ctx.set_kernel_events(ev[1], None)
    with pytest.raises(ValueError):
        ctx.set_kernel_events(torch.cuda.Event(enable_timing=True), ev[2])   # never recorded
    ctx.set_kernel_events(ev[1], ev[2])
    ev[0].record()
    call()
    ev[3].record()
    torch.cuda.synchronize()
    outer, inner = ev[0].elapsed_time(ev[3]), ev[1].elapsed_time(ev[2])
    assert 0.0 < inner <= outer
    assert ev[0].elapsed_time(ev[1]) >= 0.0 and ev[2].elapsed_time(ev[3]) >= 0.0
    # forgotten after one call: a second call leaves the events as they were
    call()
    torch.cuda.synchronize()
    assert ev[1].elapsed_time(ev[2]) == inner
    ctx.set_kernel_events(None, None)
    ctx.check()
