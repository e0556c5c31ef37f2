"""Genetic search on the device: generator, recovery of an injected source,
and equality of CUDA-graph replay with eager execution."""
import math

import numpy as np
import pytest
import torch

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


def test_ga_seeded_population_starts_from_its_seeds(api):
    # GASearch(init=...): the given starting points replace the first draws of
    # the window's population (clipped into the box); seeded with the source
    # (and a point outside the box), two generations already hold the source
    # (the best individual is kept in slot 0), while the unseeded search has
    # not found it yet
    from paper_2307_03763_gb300.ga import GASearch
    wl, src, dA, dE, box = _single_source_problem()
    ctx = api.Context(wl.T)
    args = (_cuda(dA, torch.complex128), _cuda(dE, torch.complex128), _cuda(wl.w_A, torch.float64),
            _cuda(wl.w_E, torch.float64))
    far = src.copy()
    far[0] += 100.0 / wl.T                        # outside the f0 box: clipped to its edge
    ga = GASearch(ctx, wl.windows, *args, box, pop=256, seed=11, init=[np.stack([src, far])])
    th0 = ga.th[0].cpu().numpy()
    assert np.array_equal(th0[0], np.clip(src, box[0, :8], box[0, 8:]))
    assert th0[1, 0] == box[0, 8] and np.array_equal(th0[1, 1:], np.clip(far[1:], box[0, 1:8], box[0, 9:]))
    best = ga.run(2, graph=False)[0]
    assert _overlap(wl, best, src) > 0.99
    cold = GASearch(ctx, wl.windows, *args, box, pop=256, seed=11).run(2, graph=False)[0]
    assert _overlap(wl, cold, src) < 0.9


def test_ga_step_phase_maximised_best(api):
    # gb_ga_step with dh_im on made-up inner products: window 0 (phi0 box of
    # 2 pi) ranks by sqrt(dh^2 + dh_im^2)/sqrt(hh) and rotates the best to
    # phi0 + atan2(dh_im, dh) with A_max = A |Z|/hh; window 1 (phi0 box of
    # pi) ranks by dh/sqrt(hh) and keeps phi0
    ctx = api.Context(wk.YEAR)
    rng = np.random.default_rng(5)
    pop = 300
    lo = np.array([1e-3, 0.0, -1.5, -3.0, 1e-23, 0.0, 0.0, 0.0])
    hi = np.array([1.001e-3, 1e-17, 1.5, 3.0, 1e-21, np.pi, np.pi, 2 * np.pi])
    hi1 = hi.copy()
    hi1[7] = np.pi
    box = np.stack([np.concatenate([lo, hi]), np.concatenate([lo, hi1])])
    th = lo + (np.stack([hi, hi1])[:, None, :] - lo) * rng.uniform(size=(2, pop, 8))
    th[:, :, 4] = 1e-22
    hh = rng.uniform(50.0, 200.0, size=(2, pop))
    dh = rng.uniform(-40.0, 40.0, size=(2, pop))
    dhi = rng.uniform(-40.0, 40.0, size=(2, pop))
    ib0 = int(np.argmax(np.hypot(dh[0], dhi[0]) / np.sqrt(hh[0])))
    ib1 = int(np.argmax(dh[1] / np.sqrt(hh[1])))
    # a clear winner in each window (no float ties in the ranking)
    dh[0, ib0], dhi[0, ib0] = -55.0, 60.0
    dh[1, ib1] = 70.0
    gen = torch.zeros(2, dtype=torch.int64, device=DEV)
    out, best = ctx.ga_step(2, pop, _cuda(th.reshape(-1, 8), torch.float64), _cuda(dh.ravel(), torch.float64),
                            _cuda(hh.ravel(), torch.float64), _cuda(box, torch.float64), 11, gen[0:1], gen[1:2],
                            api.GAParams(3, 0, 0.9, 0.15, 0.02), dh_im=_cuda(dhi.ravel(), torch.float64))
    best = best.cpu().numpy()
    z0 = np.hypot(dh[0, ib0], dhi[0, ib0])
    e0 = th[0, ib0].copy()
    e0[4] = min(max(e0[4] * z0 / hh[0, ib0], lo[4]), hi[4])
    e0[7] = (e0[7] + np.arctan2(dhi[0, ib0], dh[0, ib0])) % (2 * np.pi)
    e1 = th[1, ib1].copy()
    e1[4] = min(max(e1[4] * dh[1, ib1] / hh[1, ib1], lo[4]), hi[4])
    assert np.allclose(best[0], e0, rtol=1e-13, atol=1e-13 * np.abs(e0)), (best[0], e0)
    assert np.array_equal(best[1], e1), (best[1], e1)
    o = out.cpu().numpy().reshape(2, pop, 8)
    assert np.array_equal(o[:, 0], best)


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


def _draws_reference(mu, L, seed, rnd, w, i):
    """Proposal i of window w, round rnd, re-derived from the generator's definition."""
    k = [seed & 0xFFFFFFFF, seed >> 32]
    words = philox4x32_10([rnd, w, i, 0], k) + philox4x32_10([rnd, w, i, 1], k)
    u01 = lambda x: (x + 0.5) * 2.0 ** -32
    z = []
    for j in range(4):
        r = math.sqrt(-2.0 * math.log(u01(words[2 * j])))
        a = 2.0 * math.pi * u01(words[2 * j + 1])
        z += [r * math.cos(a), r * math.sin(a)]
    z = np.array(z)
    th = mu + L @ z
    lg = -0.5 * z @ z - np.log(np.diag(L)).sum() - 4 * math.log(2 * math.pi)
    lu = math.log(u01(philox4x32_10([rnd, w, i, 2], k)[0]))
    return th, lg, lu


def test_gaussian_draws_match_definition(api):
    ctx = api.Context(wk.YEAR)
    rng = np.random.default_rng(8)
    nw, n = 3, 300
    mu = rng.normal(size=(nw, 8))
    A = rng.normal(size=(nw, 8, 8)) * 0.1
    cov = A @ A.transpose(0, 2, 1) + np.eye(8)[None] * 0.5
    L = np.linalg.cholesky(cov)
    r = torch.tensor([5, 0], dtype=torch.int64, device=DEV)
    th, lg, lu = ctx.draw_gaussian(_cuda(mu, torch.float64), _cuda(L, torch.float64), n, 0x1234ABCD5678, r[0:1], r[1:2])
    assert int(r[1]) == 6
    th, lg, lu = th.cpu().numpy().reshape(nw, n, 8), lg.cpu().numpy(), lu.cpu().numpy()
    for w in range(nw):
        for i in (0, 1, 77, n - 1):
            rt, rg, ru = _draws_reference(mu[w], L[w], 0x1234ABCD5678, 5, w, i)
            assert np.allclose(th[w, i], rt, rtol=1e-13, atol=1e-13)
            assert abs(lg[w, i] - rg) < 1e-12 and abs(lu[w, i] - ru) < 1e-13
    # the draws have the requested mean and covariance
    big = ctx.draw_gaussian(_cuda(mu[:1], torch.float64), _cuda(L[:1], torch.float64), 200000, 9, r[0:1], r[1:2])[0]
    x = big.cpu().numpy()
    assert np.abs(x.mean(0) - mu[0]).max() < 6 * np.sqrt(np.diag(cov[0]).max() / 200000)
    assert np.abs(np.cov(x.T) - cov[0]).max() < 0.02 * np.abs(cov[0]).max()


def test_posterior_rounds_graph_equals_eager_and_chains_are_valid(api):
    from paper_2307_03763_gb300.posterior import PosteriorRounds
    wl, src, dA, dE, box = _single_source_problem(seed=wk.SEED_BASE + 42)
    ctx = api.Context(wl.T)
    args = (_cuda(dA, torch.complex128), _cuda(dE, torch.complex128), _cuda(wl.w_A, torch.float64),
            _cuda(wl.w_E, torch.float64))
    sig = _data.fisher_sigma(src, wl.windows[0], wl.w_A, wl.w_E, wl.T)
    cov = np.diag((3 * sig) ** 2)[None]
    a = PosteriorRounds(ctx, wl.windows, *args, src[None], cov, n=10000, seed=11).run(7, graph=False)
    b = PosteriorRounds(ctx, wl.windows, *args, src[None], cov, n=10000, seed=11).run(7, graph=True)
    assert torch.equal(a.chain, b.chain) and torch.equal(a.theta, b.theta)
    ch = b.chain[0].cpu().numpy()
    L, G, U = (x.cpu().numpy().reshape(-1) for x in (b.logL, b.log_g[0], b.log_u[0]))
    assert ch[0] == 0
    c = 0
    for i in range(1, len(ch)):
        d = (L[i] - G[i]) - (L[c] - G[c])
        if U[i] < min(0.0, d):
            c = i
        assert ch[i] == c
    assert 0 < int(b.accepted[0]) < 10000


def test_annealed_posterior_concentrates_on_the_source(api):
    # six temperatures from the T = 15 Fisher width (x 1.2), started 2 widths
    # off: the T = 1 chain sits on the source and has about the Fisher width
    from paper_2307_03763_gb300.posterior import AnnealedPosterior
    wl, src, dA, dE, box = _single_source_problem(snr=60.0, seed=wk.SEED_BASE + 43)
    ctx = api.Context(wl.T)
    args = (_cuda(dA, torch.complex128), _cuda(dE, torch.complex128), _cuda(wl.w_A, torch.float64),
            _cuda(wl.w_E, torch.float64))
    sig = _data.fisher_sigma(src, wl.windows[0], wl.w_A, wl.w_E, wl.T)
    start = src + 2.0 * sig * np.array([1, -1, 1, -1, 0.5, 1, -1, 1])
    ap = AnnealedPosterior(ctx, wl.windows, *args, start[None], np.diag(15 * (1.2 * sig) ** 2)[None], n=10000,
                           seed=5).run(graph=True)
    r = ap.rounds
    th = r.theta.view(1, r.n, 8)[0].cpu().numpy()
    states = th[r.chain[0].long().cpu().numpy()]
    mean, sd = states.mean(0), states.std(0)
    assert abs(mean[0] - src[0]) < 3 * sig[0], (mean[0], src[0], sig[0])
    assert 0.2 * sig[0] < sd[0] < 3 * sig[0], (sd[0], sig[0])
    assert int(r.accepted[0]) > 100


def test_gauss_refit_matches_its_definition(api):
    ctx = api.Context(wk.YEAR)
    rng = np.random.default_rng(17)
    nw, n = 3, 700
    scale, floor = 1.7, 1e-3
    th = rng.normal(size=(nw, n, 8)) * np.array([1e-9, 1e-17, 0.1, 0.2, 1e-23, 0.3, 0.1, 0.5]) \
        + np.array([3e-3, 1e-16, 0.2, 1.0, 1e-22, 1.0, 0.5, 2.0])
    ch = np.zeros((nw, n), np.int32)
    for w in range(nw):
        c = 0
        for i in range(1, n):
            if rng.uniform() < 0.3:
                c = i
            ch[w, i] = c
    A = rng.normal(size=(nw, 8, 8)) * 0.3
    L0 = np.linalg.cholesky(A @ A.transpose(0, 2, 1) + np.eye(8)) * np.array([1e-8, 1e-16, 1, 1, 1e-22, 1, 1, 1])[:, None]
    L0 = np.tril(L0)
    mu = torch.empty((nw, 8), dtype=torch.float64, device=DEV)
    chol = torch.empty((nw, 8, 8), dtype=torch.float64, device=DEV)
    B = rng.normal(size=(nw, 8, 8)) * 0.2
    Lp = np.tril(np.linalg.cholesky(B @ B.transpose(0, 2, 1) + np.eye(8))) * np.array(
        [1e-8, 1e-16, 1, 1, 1e-22, 1, 1, 1])[:, None]
    chol.copy_(_cuda(Lp, torch.float64))
    inflate, kappa = 1.3, 40.0
    ctx.gauss_refit(_cuda(th.reshape(-1, 8), torch.float64), _cuda(ch, torch.int32), _cuda(L0, torch.float64),
                    scale, inflate, kappa, floor, out=(mu, chol))
    mu, chol = mu.cpu().numpy(), chol.cpu().numpy()
    for w in range(nw):
        st = th[w][ch[w]]
        m = st.mean(0)
        u = np.sum(ch[w][1:] == np.arange(1, n))
        g = u / (u + kappa)
        C = scale * (g * inflate * np.cov(st.T, ddof=1) + (1 - g) * Lp[w] @ Lp[w].T)
        Li = np.linalg.inv(L0[w])
        M = Li @ C @ Li.T
        d = np.maximum(1.0, np.sqrt(np.diag(M) * floor))
        M = M / np.outer(d, d) + floor * np.eye(8)
        ref = L0[w] @ np.linalg.cholesky(M)
        assert np.allclose(mu[w], m, rtol=1e-12, atol=0)
        assert np.allclose(chol[w], ref, rtol=1e-9, atol=1e-9 * np.abs(ref).max(axis=1, keepdims=True).max())
        assert np.all(np.triu(chol[w], 1) == 0)


def test_annealed_ladder_graph_replay_equals_eager(api):
    from paper_2307_03763_gb300.posterior import AnnealedPosterior
    wl, src, dA, dE, box = _single_source_problem(snr=40.0, seed=wk.SEED_BASE + 44)
    ctx = api.Context(wl.T)
    args = (_cuda(dA, torch.complex128), _cuda(dE, torch.complex128), _cuda(wl.w_A, torch.float64),
            _cuda(wl.w_E, torch.float64))
    sig = _data.fisher_sigma(src, wl.windows[0], wl.w_A, wl.w_E, wl.T)
    a = AnnealedPosterior(ctx, wl.windows, *args, src[None], np.diag((10 * sig) ** 2)[None], n=4000, seed=9)
    b = AnnealedPosterior(ctx, wl.windows, *args, src[None], np.diag((10 * sig) ** 2)[None], n=4000, seed=9)
    a.run()
    a.run()                  # the second ladder
    b.run(graph=True)        # eager ladder + capture
    b.run(graph=True)        # replay: the second ladder
    assert torch.equal(a.rounds.chain, b.rounds.chain) and torch.equal(a.rounds.theta, b.rounds.theta)
    assert torch.equal(a.rounds.chol, b.rounds.chol)


def test_newton_polish_reaches_the_maximum(api):
    # noise-free data: the likelihood peaks at the source; start one Fisher
    # width away in every parameter
    from paper_2307_03763_gb300.autograd import newton_polish
    wl, src, _, _, _ = _single_source_problem(snr=50.0, seed=wk.SEED_BASE + 45)
    ctx = api.Context(wl.T)
    hA, hE = _data.template_on_window(src, *wl.windows[0][:3], wl.T)
    args = (_cuda(hA, torch.complex128), _cuda(hE, torch.complex128), _cuda(wl.w_A, torch.float64),
            _cuda(wl.w_E, torch.float64))
    sig = _data.fisher_sigma(src, wl.windows[0], wl.w_A, wl.w_E, wl.T)
    start = src + sig * np.array([1, -1, 1, -1, 0.5, 1, -1, 1])
    l0 = ctx.loglik(wl.windows[:1], *args, _cuda(start[None], torch.float64), prec="fp64")[0]
    th, L = newton_polish(ctx, wl.windows, *args, _cuda(start[None], torch.float64), iters=10, prec="fp64")
    th = th.cpu().numpy()[0]
    # the maximum is logL = 0; f0, fdot and the sky position converge, while
    # (A, iota, psi, phi0) move along their curved degeneracy valley
    assert float(L[0]) > max(float(l0[0]), -0.1), (float(l0[0]), float(L[0]))
    assert np.all(np.abs(th[:4] - src[:4]) < 0.05 * sig[:4]), (th - src) / sig
