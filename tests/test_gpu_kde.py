"""The paired KDE proposals of Alg. 4 (gb_kde_build / gb_kde_draw) against the
oracle, and the annealed posterior the paper describes (uniform start in the
reduced box, KDE proposals afterwards) on an injected source."""
import math

import numpy as np
import pytest
import torch

from oracle import kde as okde
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
    return torch.as_tensor(np.ascontiguousarray(x)).to(DEV, dtype)


def _chains(rng, nw, n, p_acc):
    ch = np.zeros((nw, n), np.int32)
    for w in range(nw):
        c = 0
        for i in range(1, n):
            if rng.uniform() < p_acc[w]:
                c = i
            ch[w, i] = c
    return ch


def _boxes(rng, nw):
    lo = np.array([3e-3, 0.0, -0.3, 0.5, 1e-22, 0.4, 0.9, 1.0])
    wid = np.array([4e-9, 2e-16, 0.2, 0.3, 4e-23, 0.8, 2e-3, 4e-3])
    b = np.empty((nw, 16))
    for w in range(nw):
        l = lo * (1 + 0.1 * rng.uniform(size=8))
        b[w, :8], b[w, 8:] = l, l + wid * (0.5 + rng.uniform(size=8))
    return b


@pytest.mark.parametrize("grid", [64, 20, 2])
def test_kde_build_matches_oracle(api, grid):
    # three windows: chains that move often, rarely and never (no smoothing);
    # proposals spread over the box and partly outside it (clamped cells)
    ctx = api.Context(wk.YEAR)
    rng = np.random.default_rng(23 + grid)
    nw, n = 3, 1500
    box = _boxes(rng, nw)
    lo, hi = box[:, :8], box[:, 8:]
    centre, width = (lo + hi) / 2, hi - lo
    th = centre[:, None, :] + width[:, None, :] * rng.normal(0.0, 0.25, size=(nw, n, 8))
    ch = _chains(rng, nw, n, [0.4, 0.02, 0.0])
    cdf = torch.empty((nw, 3, grid * grid), dtype=torch.float64, device=DEV)
    ext = torch.empty((nw, 3, 4), dtype=torch.float64, device=DEV)
    ctx.kde_build(_cuda(th.reshape(-1, 8), torch.float64), _cuda(ch, torch.int32), _cuda(box, torch.float64), grid,
                  0.01, out=(cdf, ext))
    got, gext = cdf.cpu().numpy(), ext.cpu().numpy()
    for w in range(nw):
        ref, rext = okde.build_window(th[w], ch[w], lo[w], hi[w], grid, 0.01)
        assert np.allclose(gext[w], rext, rtol=1e-12, atol=0), (w, gext[w], rext)
        assert np.abs(got[w] - ref).max() < 2e-6, (w, np.abs(got[w] - ref).max())
        assert np.all(np.diff(got[w], axis=1) > 0) and np.allclose(got[w][:, -1], 1.0, atol=1e-12)


def test_kde_draw_matches_oracle(api):
    # tables from the oracle (one smoothed, one flat, one peaked), draws
    # compared proposal by proposal with the oracle fed the same Philox words
    ctx = api.Context(wk.YEAR)
    rng = np.random.default_rng(31)
    nw, n, G = 2, 3000, 16
    box = _boxes(rng, nw)
    lo, hi = box[:, :8], box[:, 8:]
    th = (lo + hi)[:, None, :] / 2 + (hi - lo)[:, None, :] * rng.normal(0.0, 0.2, size=(nw, n, 8))
    ch = _chains(rng, nw, n, [0.3, 0.01])
    built = [okde.build_window(th[w], ch[w], lo[w], hi[w], G, 0.02) for w in range(nw)]
    C = np.stack([b[0] for b in built])
    E = np.stack([b[1] for b in built])
    C[1, 1] = okde.cumulative(okde.flat_grid(G))
    E[1, 1] = okde.box_extents(lo[1], hi[1])[1]
    seed = 0x5EED0000C0FFEE
    r = torch.tensor([41, 0], dtype=torch.int64, device=DEV)
    t, lg, lu = ctx.kde_draw(_cuda(box, torch.float64), G, _cuda(C, torch.float64), _cuda(E, torch.float64), n, seed,
                             r[0:1], r[1:2])
    assert int(r[1]) == 42
    t, lg, lu = t.cpu().numpy().reshape(nw, n, 8), lg.cpu().numpy(), lu.cpu().numpy()
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for w in range(nw):
        for i in list(range(0, n, 97)) + [n - 1]:
            words = sum((philox4x32_10([41, w, i, b], key) for b in range(3)), [])
            rt, rg, ru = okde.draw(C[w], E[w], lo[w], hi[w], G, words)
            assert np.allclose(t[w, i], rt, rtol=1e-15, atol=0), (w, i, t[w, i], rt)
            assert abs(lg[w, i] - rg) <= 1e-12 * abs(rg) and abs(lu[w, i] - ru) <= 1e-13
    # every draw inside its box
    assert np.all(t >= lo[:, None, :]) and np.all(t <= hi[:, None, :])


def test_kde_draw_flat_table_is_uniform(api):
    ctx = api.Context(wk.YEAR)
    G = 8
    box = np.concatenate([np.zeros(8), np.arange(1, 9, dtype=float)])[None]
    C = np.stack([okde.cumulative(okde.flat_grid(G))] * 3)[None]
    E = okde.box_extents(box[0, :8], box[0, 8:])[None]
    r = torch.tensor([0, 0], dtype=torch.int64, device=DEV)
    t, lg, _ = ctx.kde_draw(_cuda(box, torch.float64), G, _cuda(C, torch.float64), _cuda(E, torch.float64), 100000, 3,
                            r[0:1], r[1:2])
    u = t.cpu().numpy() / np.arange(1, 9)
    assert np.allclose(lg.cpu().numpy(), -math.log(math.factorial(8)), rtol=1e-12)
    assert np.abs(u.mean(0) - 0.5).max() < 0.005 and np.abs(u.var(0) - 1 / 12).max() < 0.002


def _posterior_problem(api, snr, seed):
    wl = wk.tiny_window(seed=seed, n_cand=1)
    src = wl.sources[0][0].copy()
    src[4] *= snr / _data.unit_snr(src, wl.windows[0], wl.w_A, wl.w_E, wl.T)
    dA, dE = _data.inject(wl, [[src]])
    sig = _data.fisher_sigma(src, wl.windows[0], wl.w_A, wl.w_E, wl.T)
    k0, W = wl.windows[0][0], wl.windows[0][1]
    plo = np.array([k0 / wl.T, 0.0, -np.pi / 2, -np.pi, 1e-24, 0.0, 0.0, 0.0])
    phi = np.array([(k0 + W) / wl.T, 2 * src[1] + 1e-17, np.pi / 2, np.pi, 1e-20, np.pi, np.pi, 2 * np.pi])
    args = (_cuda(dA, torch.complex128), _cuda(dE, torch.complex128), _cuda(wl.w_A, torch.float64),
            _cuda(wl.w_E, torch.float64))
    return wl, src, sig, plo, phi, args


def test_kde_posterior_concentrates_on_the_source(api):
    # the paper's ladder from the uniform reduced box: at T = 1 the chain's
    # states sit on the source with about the Fisher width
    from paper_2307_03763_gb300.posterior import KDEPosterior, reduced_box
    wl, src, sig, plo, phi, args = _posterior_problem(api, 60.0, wk.SEED_BASE + 44)
    ctx = api.Context(wl.T)
    box = reduced_box(src[None], sig[None], plo, phi)
    kp = KDEPosterior(ctx, wl.windows, *args, box, n=10000, seed=9).run(graph=True)
    th = kp.theta.view(kp.n, 8).cpu().numpy()
    states = th[kp.chain[0].long().cpu().numpy()]
    mean, sd = states.mean(0), states.std(0)
    for d in (0, 2, 3):   # the noise moves the posterior mean by about a Fisher width
        assert abs(mean[d] - src[d]) < 3 * sig[d], (d, mean[d], src[d], sig[d])
        assert 0.2 * sig[d] < sd[d] < 1.5 * sig[d], (d, sd[d], sig[d])
    assert int(kp.accepted[0]) > 300, int(kp.accepted[0])
    assert np.all(states >= box[0, :8]) and np.all(states <= box[0, 8:])


def test_kde_ladder_graph_replay_equals_eager(api):
    from paper_2307_03763_gb300.posterior import KDEPosterior, reduced_box
    wl, src, sig, plo, phi, args = _posterior_problem(api, 40.0, wk.SEED_BASE + 45)
    ctx = api.Context(wl.T)
    box = reduced_box(src[None], sig[None], plo, phi)
    for temps in ((15, 10, 5, 3, 2, 1), (5, 2, 1)):   # even and odd ladders
        a = KDEPosterior(ctx, wl.windows, *args, box, n=4000, seed=13, temperatures=temps)
        b = KDEPosterior(ctx, wl.windows, *args, box, n=4000, seed=13, temperatures=temps)
        for _ in range(3):
            a.run(graph=False)
            b.run(graph=True)
            assert torch.equal(a.chain, b.chain) and torch.equal(a.theta, b.theta)
        # each posterior draws new numbers
        first = a.theta.clone()
        a.run(graph=False)
        assert not torch.equal(first, a.theta)
