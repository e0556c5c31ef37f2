"""The T channel (Eq. 5; used above f*/2, Sec. II) through the C ABI against
the oracle: FP64 templates and likelihoods to 1e-10, the mixed likelihood to
1e-5 of <h|h>, windows below f*/2 unchanged from gb_loglik."""
import math

import numpy as np
import pytest
import torch

from oracle import gb as ogb
from paper_2307_03763_gb300 import workloads as wk

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
T = wk.YEAR


@pytest.fixture(scope="module")
def ctx():
    from paper_2307_03763_gb300 import api, build
    build.build()
    return api.Context(T)


def _c(x, dt):
    return torch.as_tensor(np.ascontiguousarray(x)).to(DEV, dt)


def _problem(seed, specs, n_cand):
    """Windows (f0, N) with an injected source each, noise and weights per channel."""
    rng = np.random.default_rng(seed)
    wins, th_all, data, weights = [], [], [[], [], []], [[], [], []]
    off = coff = 0
    for f0, N in specs:
        src = wk.source(f0, float(wk.chirp_fdot(f0, 0.5)), 1e-22, rng)
        q = int(ogb.carrier_bin(torch.tensor([src[0]]), torch.tensor([src[1]]), T)[0][0])
        k0, W = q - N // 2 + 3, N
        _, hA, hE, hT = ogb.template_aet(torch.tensor(src[None]), N, T)
        for c, (h, wv) in enumerate(zip((hA, hE, hT), (1e41, 1e41, 3e41))):
            x = np.zeros(W, np.complex128)
            x[:N - 3] = h[0].numpy()[3:]
            sd = math.sqrt(T / (4 * wv))
            data[c].append(x + (rng.normal(size=W) + 1j * rng.normal(size=W)) * sd)
            weights[c].append(np.full(W, wv) * (1 + 0.1 * rng.uniform(size=W)))
        half = np.array([2 / T, abs(src[1]), 0.05, 0.05, 0.1 * src[4], 0.05, 0.05, 0.2])
        th_all.append(wk.uniform_box(src, half, n_cand, rng))
        wins.append((k0, W, N, off, coff, n_cand))
        off += W
        coff += n_cand
    d = [np.concatenate(x) for x in data]
    w = [np.concatenate(x) for x in weights]
    return wins, np.concatenate(th_all), d, w


SPECS = [(6e-3, 256), (11e-3, 512), (16e-3, 1024), (9.8e-3, 256)]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_waveform_aet_matches_oracle(ctx, prec):
    # FP64 to 1e-10 of each channel's peak; mixed to 2e-6 of A's peak (the
    # float response; T itself is 0.01-1% of A below 20 mHz)
    rng = np.random.default_rng(3)
    th = np.stack([wk.source(f, 1e-16, 1e-22, rng) for f in (2e-3, 12e-3, 17e-3)])
    for N in (64, 256, 1024):
        hA, hE, hT, q = ctx.waveform_aet(_c(th, torch.float64), N, prec=prec)
        oq, oA, oE, oT = ogb.template_aet(torch.tensor(th), N, T)
        assert torch.equal(q.cpu(), oq)
        peakA = oA.abs().max(dim=1).values
        for g, o in ((hA, oA), (hE, oE), (hT, oT)):
            g = g.cpu()
            if prec == "fp64":
                assert ((g - o).abs().max(dim=1).values <= 1e-10 * o.abs().max(dim=1).values + 1e-300).all()
            else:
                assert ((g - o).abs().max(dim=1).values <= 2e-6 * peakA).all()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_loglik_aet_matches_oracle(ctx, prec):
    wins, th, d, w = _problem(7, SPECS, 24)
    assert [ogb.uses_t(k0, T) for k0, *_ in wins] == [False, True, True, True]
    args = [_c(x, torch.complex128) for x in d] + [_c(x, torch.float64) for x in w]
    g = [x.cpu() for x in ctx.loglik_aet(wins, *args, _c(th, torch.float64), prec=prec)]
    o = ogb.loglik_aet(wins, *d, *w, th, T)
    if prec == "fp64":
        scale = max(1.0, float(o[2].abs().max()))
        assert float((g[0] - o[0]).abs().max()) <= 1e-10 * float(o[0].abs().max())
        assert float((g[1] - o[1]).abs().max()) <= 1e-10 * scale
        assert float((g[2] - o[2]).abs().max()) <= 1e-10 * scale
    else:
        rel = (g[0] - o[0]).abs() / torch.clamp(o[2].abs(), min=1.0)
        assert float(rel.max()) < 1e-5, float(rel.max())
    # the window below f*/2 is the plain A/E likelihood
    a = [x.cpu() for x in ctx.loglik(wins[:1], args[0], args[1], args[3], args[4], _c(th, torch.float64), prec=prec)]
    n0 = wins[0][5]
    assert torch.equal(a[0][:n0], g[0][:n0])


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_loglik_aet_every_template_length(ctx, prec):
    # T windows at every N (the mixed kernel's N = 32, 64, 128 branches take
    # the other second-stage forms of the transform), ragged candidate counts
    specs = [(10.0e-3, 32), (10.5e-3, 64), (11e-3, 128), (12e-3, 256), (13e-3, 512), (14e-3, 1024)]
    wins, th, d, w = _problem(11, specs, 9)
    wins = [(k0, W, N, doff, coff, nc) for (k0, W, N, doff, coff, nc) in wins]
    assert all(ogb.uses_t(k0, T) for k0, *_ in wins)
    args = [_c(x, torch.complex128) for x in d] + [_c(x, torch.float64) for x in w]
    g = [x.cpu() for x in ctx.loglik_aet(wins, *args, _c(th, torch.float64), prec=prec)]
    o = ogb.loglik_aet(wins, *d, *w, th, T)
    if prec == "fp64":
        assert float((g[0] - o[0]).abs().max()) <= 1e-10 * float(o[0].abs().max())
        assert float((g[2] - o[2]).abs().max()) <= 1e-10 * max(1.0, float(o[2].abs().max()))
    else:
        rel = (g[0] - o[0]).abs() / torch.clamp(o[2].abs(), min=1.0)
        assert float(rel.max()) < 1e-5, float(rel.max())


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_loglik_aet_edge_windows(ctx, prec):
    # a T window whose templates fall outside it, one with W = 0 and one with
    # no candidates, next to an ordinary one
    wins, th, d, w = _problem(12, [(12e-3, 256), (13e-3, 256)], 6)
    (k0a, Wa, Na, da_, ca, na), (k0b, Wb, Nb, db, cb, nb) = wins
    wins = [(k0a, Wa, Na, da_, ca, na), (k0b + 10 * Nb, Wb, Nb, db, cb, nb), (k0b, 0, Nb, db, cb, 0),
            (k0a, Wa, Na, da_, cb + nb, 0)]
    args = [_c(x, torch.complex128) for x in d] + [_c(x, torch.float64) for x in w]
    g = [x.cpu() for x in ctx.loglik_aet(wins, *args, _c(th, torch.float64), prec=prec)]
    o = ogb.loglik_aet(wins, *d, *w, th, T)
    tol = 1e-10 if prec == "fp64" else 1e-5
    scale = torch.clamp(o[2].abs(), min=1.0)
    assert float(((g[0] - o[0]).abs() / torch.clamp(o[0].abs(), min=1.0)).max()) < tol
    assert float(((g[2] - o[2]).abs() / scale).max()) < tol
    assert float(g[2][na:].abs().max()) == 0.0          # no template inside: <h|h> = 0


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_loglik_grad_aet_matches_oracle(ctx, prec):
    # the adjoint gradient with T against autodiff of the oracle's three-channel
    # likelihood (natural units): FP64 to 1e-9, mixed to 1e-4 of the gradient's
    # norm; windows below f*/2 and at N = 256, 512, 1,024 above it
    specs = [(6e-3, 256), (11e-3, 512), (12e-3, 256), (16e-3, 1024)]
    wins, th, d, w = _problem(13, specs, 3)
    args = [_c(x, torch.complex128) for x in d] + [_c(x, torch.float64) for x in w]
    lg, gg = (x.cpu() for x in ctx.loglik_grad_aet(wins, *args, _c(th, torch.float64), prec=prec))
    lo, go = ogb.loglik_grad_aet(wins, *d, *w, th, T)
    s = torch.tensor([1 / T, 1 / T ** 2, 1, 1, 1, 1, 1, 1], dtype=torch.float64)
    tol = 1e-9 if prec == "fp64" else 1e-4
    for b in range(th.shape[0]):
        sb = s.clone()
        sb[4] = th[b, 4]
        gn, on = gg[b] * sb, go[b] * sb
        assert float((gn - on).abs().max()) <= tol * float(on.abs().sum()), (prec, b, gn, on)
    ltol = 1e-10 if prec == "fp64" else 1e-5
    assert float(((lg - lo).abs() / lo.abs().clamp(min=1.0)).max()) < ltol
    # without T data it is the A/E gradient
    g2 = ctx.loglik_grad(wins[:1], args[0], args[1], args[3], args[4], _c(th, torch.float64), prec=prec)[1].cpu()
    n0 = wins[0][5]
    assert torch.equal(g2[:n0], gg[:n0])


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_loglik_phase_aet_is_dh_at_a_quarter_turn(ctx, prec):
    # with T, dh_im(theta) = <d|h> over A, E and T at phi0 + pi/2
    specs = [(6e-3, 256), (11e-3, 512), (12e-3, 256)]
    wins, th, d, w = _problem(14, specs, 10)
    args = [_c(x, torch.complex128) for x in d] + [_c(x, torch.float64) for x in w]
    lp, dp, dip, hp = (x.cpu() for x in ctx.loglik_phase_aet(wins, *args, _c(th, torch.float64), prec=prec))
    la, da, ha = (x.cpu() for x in ctx.loglik_aet(wins, *args, _c(th, torch.float64), prec=prec))
    tq = th.copy()
    tq[:, 7] += np.pi / 2
    _, oq, ohh = ogb.loglik_aet(wins, *d, *w, tq, T)
    scale = torch.clamp(ohh.abs(), min=1.0)
    tol = 1e-10 if prec == "fp64" else 1e-5
    assert float(((dip - oq).abs() / scale).max()) < tol
    # the other outputs are those of loglik_aet
    for a, b in ((lp, la), (dp, da), (hp, ha)):
        assert float(((a - b).abs() / scale).max()) < tol


def test_t_channel_argument_errors(ctx):
    from paper_2307_03763_gb300 import api
    rng = np.random.default_rng(9)
    th = _c(np.stack([wk.source(12e-3, 1e-16, 1e-22, rng)]), torch.float64)
    with pytest.raises(api.GBError):
        ctx.waveform_aet(th, 100)                      # N not a power of two
    h = torch.empty((1, 256), dtype=torch.complex128, device=DEV)
    q = torch.empty(1, dtype=torch.int64, device=DEV)
    rc = api.lib().gb_waveform_aet(ctx._h, 7, api._ptr(th), 1, 256, api._ptr(h), api._ptr(h),
                                   api._ptr(h), api._ptr(q), None)
    assert rc != 0                                     # unknown precision
