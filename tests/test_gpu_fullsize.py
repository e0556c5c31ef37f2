"""Parity at full workload sizes, in the launch configuration the benchmark
times (autotuned shapes, one launch over every window), on sampled rows the
oracle computes one by one.

* band workload: 512 windows over 0.3-20 mHz at T = 1 yr, N = 32..1024,
  2,000-20,000 candidates per window (about 5.6M per launch), both precisions;
* population workload: 64 windows of N = 256 at T = 2 yr, 4,096 candidates
  each, the mixed-precision adjoint gradient.
"""
import numpy as np
import pytest
import torch

from oracle import gb as ogb
from paper_2307_03763_gb300 import workloads as wk
from tests import _data

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module")
def api():
    from paper_2307_03763_gb300 import api, build
    build.build()
    return api


def _cuda(x, dtype):
    return torch.as_tensor(np.ascontiguousarray(x)).to(device=DEV, dtype=dtype)


def _sample(wl, rng, per_window):
    """First, last and per_window random rows of every window; the oracle's
    sub-windows over them."""
    rows = []
    for (k0, W, N, doff, coff, nc) in wl.windows:
        rows += [coff, coff + nc - 1] + list(coff + rng.choice(nc, per_window, replace=False))
    rows = np.array(sorted(set(rows)))
    sub, off = [], 0
    for (k0, W, N, doff, coff, nc) in wl.windows:
        n = int(((rows >= coff) & (rows < coff + nc)).sum())
        sub.append((k0, W, N, doff, off, n))
        off += n
    return rows, sub


def test_band_workload_full_launch_sampled(api):
    wl = wk.band_windows()
    assert len(wl.windows) == 512 and wl.n_cand > 5_000_000
    ctx = api.Context(wl.T)
    dA, dE = _data.inject(wl)
    args = (_cuda(dA, torch.complex128), _cuda(dE, torch.complex128), _cuda(wl.w_A, torch.float64),
            _cuda(wl.w_E, torch.float64))
    theta = _cuda(wl.theta, torch.float64)
    ctx.autotune(wl.windows, *args, theta, prec="mixed", reps=2)
    gmx = [x.cpu() for x in ctx.loglik(wl.windows, *args, theta, prec="mixed")]
    g64 = [x.cpu() for x in ctx.loglik(wl.windows, *args, theta, prec="fp64")]
    del theta
    rows, sub = _sample(wl, np.random.default_rng(17), 2)
    o = ogb.loglik(sub, dA, dE, wl.w_A, wl.w_E, wl.theta[rows], wl.T)
    idx = torch.tensor(rows)
    scale = torch.clamp(o[2].abs(), min=1.0)
    for g, a in zip(g64, o):
        rel = (g[idx] - a).abs() / torch.maximum(scale, a.abs())
        assert float(rel.max()) <= 1e-10, float(rel.max())
    rel = (gmx[0][idx] - o[0]).abs() / scale
    assert float(rel.max()) < 1e-5, float(rel.max())
    # every row of the launch is finite
    assert bool(torch.isfinite(gmx[0]).all()) and bool(torch.isfinite(g64[0]).all())


def test_population_gradient_full_launch_sampled(api):
    wl = wk.population_windows()
    assert len(wl.windows) == 64 and wl.n_cand == 64 * 4096
    ctx = api.Context(wl.T)
    dA, dE = _data.inject(wl)
    args = (_cuda(dA, torch.complex128), _cuda(dE, torch.complex128), _cuda(wl.w_A, torch.float64),
            _cuda(wl.w_E, torch.float64), _cuda(wl.theta, torch.float64))
    lg, gg = (x.cpu() for x in ctx.loglik_grad(wl.windows, *args, prec="mixed"))
    rows, sub = _sample(wl, np.random.default_rng(19), 1)
    lo, go = ogb.loglik_grad(sub, dA, dE, wl.w_A, wl.w_E, wl.theta[rows], wl.T)
    worst = 0.0
    for i, r in enumerate(rows):
        # natural parameter units: f0 in bins, fdot in bins per T, A relative
        s = torch.tensor([1 / wl.T, 1 / wl.T ** 2, 1, 1, wl.theta[r, 4], 1, 1, 1], dtype=torch.float64)
        gn, on = gg[r] * s, go[i] * s
        worst = max(worst, float((gn - on).abs().max()) / float(on.abs().sum()))
    assert worst <= 1e-4, worst
    o = ogb.loglik(sub, dA, dE, wl.w_A, wl.w_E, wl.theta[rows], wl.T)
    assert float(((lg[torch.tensor(rows)] - o[0]).abs() / torch.clamp(o[2].abs(), min=1.0)).max()) < 1e-5
    assert bool(torch.isfinite(gg).all())
