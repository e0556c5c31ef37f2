"""Genetic search on the device: generator, recovery of an injected source,
and equality of CUDA-graph replay with eager execution."""
import math

import numpy as np
import pytest
import torch

from oracle import gb as ogb
from paper_2307_03763_gb300 import workloads as wk
from tests import _data
from tests._philox import philox4x32_10

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def api():
    from paper_2307_03763_gb300 import api, build
    build.build()
    return api


def _cuda(x, dtype):
    return torch.as_tensor(np.ascontiguousarray(x)).to(device=DEV, dtype=dtype)


def test_philox_matches_reference(api):
    ctx = api.Context(wk.YEAR)
    for seed in (0, 123456789, 0xDEADBEEFCAFEF00D):
        out = ctx.philox(seed, 257).cpu().numpy()
        for i in (0, 1, 31, 32, 255, 256):
            assert list(out[i]) == philox4x32_10([i, 0, 0, 0], [seed & 0xFFFFFFFF, seed >> 32])


def _single_source_problem(snr=60.0, seed=wk.SEED_BASE + 40):
    wl = wk.tiny_window(seed=seed, n_cand=1)
    src = wl.sources[0][0].copy()
    src[4] *= snr / _data.unit_snr(src, wl.windows[0], wl.w_A, wl.w_E, wl.T)
    dA, dE = _data.inject(wl, [[src]])
    T = wl.T
    lo = np.array([src[0] - 6 / T, 0.0, -np.pi / 2, -np.pi, 0.3 * src[4], 0.0, 0.0, 0.0])
    hi = np.array([src[0] + 6 / T, 2 * src[1], np.pi / 2, np.pi, 3.0 * src[4], np.pi, np.pi, 2 * np.pi])
    return wl, src, dA, dE, np.concatenate([lo, hi])[None, :]


def _overlap(wl, a, b):
    """Eq. 20 overlap of two parameter sets on the window (oracle templates)."""
    k0, W, N, doff, _, _ = wl.windows[0]
    ha = _data.template_on_window(a, k0, W, N, wl.T)
    hb = _data.template_on_window(b, k0, W, N, wl.T)
    ip = lambda x, y: (4 / wl.T) * sum(np.sum(w * (p * q.conj()).real) for w, p, q in
                                       ((wl.w_A, x[0], y[0]), (wl.w_E, x[1], y[1])))
    return ip(ha, hb) / math.sqrt(ip(ha, ha) * ip(hb, hb))


def test_ga_recovers_an_injected_source(api):
    from paper_2307_03763_gb300.ga import GASearch
    wl, src, dA, dE, box = _single_source_problem()
    ctx = api.Context(wl.T)
    args = (_cuda(dA, torch.complex128), _cuda(dE, torch.complex128), _cuda(wl.w_A, torch.float64),
            _cuda(wl.w_E, torch.float64))
    ga = GASearch(ctx, wl.windows, *args, box, pop=4096, seed=7)
    best = ga.run(200, graph=True)[0]
    rho = ga.best_snr()[0]
    ovl = _overlap(wl, best, src)
    assert ovl > 0.9, (ovl, rho, best, src)
    assert rho > 0.8 * 60.0


def test_ga_graph_replay_equals_eager(api):
    from paper_2307_03763_gb300.ga import GASearch
    wl, src, dA, dE, box = _single_source_problem(seed=wk.SEED_BASE + 41)
    ctx = api.Context(wl.T)
    args = (_cuda(dA, torch.complex128), _cuda(dE, torch.complex128), _cuda(wl.w_A, torch.float64),
            _cuda(wl.w_E, torch.float64))
    a = GASearch(ctx, wl.windows, *args, box, pop=1024, seed=3)
    b = GASearch(ctx, wl.windows, *args, box, pop=1024, seed=3)
    ba = a.run(21, graph=False)
    bb = b.run(21, graph=True)
    assert np.array_equal(ba, bb)
    assert torch.equal(a.th[a.cur], b.th[b.cur])
