"""Multi-signal SNR (Eq. 11), its Gram matrix and the match metrics (Eqs. 19-20)
through gb_snr_multi, against the oracle (FP64, 1e-10 of the scale <h|h>)."""
import math

import numpy as np
import pytest
import torch

from oracle import gb as ogb
from paper_2307_03763_gb300 import workloads as wk
from tests import _data

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
T2 = 2 * wk.YEAR


def _cuda(x, dtype):
    return torch.as_tensor(np.ascontiguousarray(x)).to(device=DEV, dtype=dtype)


@pytest.fixture(scope="module")
def api():
    from paper_2307_03763_gb300 import api, build
    build.build()
    return api


def _multi_workload(rng):
    """Windows of N = 32 ... 1024 holding 0 to 5 sources each: overlapping
    (a few bins apart), disjoint (far apart in a wide window), partly outside."""
    T = T2
    specs, counts, srcs, th = [], [], [], []
    plan = [(32, 0.7e-3, 0, 32), (64, 1.2e-3, 2, 64), (128, 2.0e-3, 3, 128), (128, 2.6e-3, 1, 128),
            (256, 4.0e-3, 5, 256), (512, 9.0e-3, 4, 512), (1024, 1.5e-2, 2, 1024), (128, 3.3e-3, 2, 1024),
            (256, 5.0e-3, 3, 200)]
    for N, f0, K, W in plan:
        kc = int(round(f0 * T))
        s = []
        for k in range(K):
            spread = 300.0 if W > 4 * N else 4.0
            f = f0 + (k - (K - 1) / 2) * spread / T + rng.uniform(-0.3, 0.3) / T
            s.append(wk.source(f, float(wk.chirp_fdot(f, 0.4)), math.exp(rng.uniform(math.log(1e-22), math.log(8e-22))),
                               rng))
        specs.append((kc - W // 2, W, N))
        counts.append(K)
        srcs.append(s)
        th += s
    wins, _, _ = wk.layout(specs, counts)
    nA, nE, wA, wE = wk.noise_and_weights(wins, T, rng)
    wl = wk.Workload("multi", T, wins, nA, nE, wA, wE, srcs, np.array(th).reshape(-1, 8))
    return wl


def test_snr_multi_matches_oracle(api):
    rng = np.random.default_rng(51)
    wl = _multi_workload(rng)
    ctx = api.Context(wl.T)
    dA, dE = _data.inject(wl)
    rho, G, b = ctx.snr_multi(wl.windows, _cuda(dA, torch.complex128), _cuda(dE, torch.complex128),
                              _cuda(wl.w_A, torch.float64), _cuda(wl.w_E, torch.float64),
                              _cuda(wl.theta, torch.float64))
    rho, G, b = rho.cpu(), G.cpu(), b.cpu()
    orho, oG, ob = ogb.snr_multi(wl.windows, dA, dE, wl.w_A, wl.w_E, wl.theta, wl.T)
    for w, (k0, W, N, doff, coff, nc) in enumerate(wl.windows):
        if nc == 0:
            assert math.isnan(float(rho[w]))
            continue
        scale = float(oG[w].abs().max())
        assert float((G[w, :nc, :nc] - oG[w]).abs().max()) <= 1e-10 * scale, w
        assert float((b[coff:coff + nc] - ob[coff:coff + nc]).abs().max()) <= 1e-10 * max(scale, 1.0), w
        assert abs(float(rho[w] - orho[w])) <= 1e-10 * max(1.0, abs(float(orho[w]))), w
    # overlapping windows have cross terms, the disjoint one none
    assert abs(float(G[4, 0, 1])) > 1e-3 * float(G[4, 0, 0])
    assert float(G[7, 0, 1]) == 0.0
    ctx.close()


def test_match_metrics_from_the_gram_matrix(api):
    # recovered sources near injected ones (small perturbations, a doubled
    # amplitude, a phase flip): delta and O from gb_snr_multi's 2 x 2 Gram
    # matrices against the oracle's literal Eqs. 19-20
    rng = np.random.default_rng(52)
    T = T2
    pairs, specs = [], []
    for N, f0 in [(64, 1.1e-3), (128, 2.2e-3), (256, 4.4e-3), (512, 1.1e-2)]:
        inj = wk.source(f0, float(wk.chirp_fdot(f0, 0.5)), 4e-22, rng)
        for kind in range(4):
            rec = inj.copy()
            if kind == 0:
                rec[0] += 0.2 / T
                rec[2:4] += 0.02
            elif kind == 1:
                rec[4] *= 2.0
            elif kind == 2:
                rec[7] += math.pi
            else:
                rec[0] += 1.5 / T
            kc = int(round(f0 * T))
            specs.append((kc - N // 2, N, N))
            pairs.append((rec, inj))
    wins, _, _ = wk.layout(specs, [2] * len(specs))
    _, _, wA, wE = wk.noise_and_weights(wins, T, rng)
    th = np.concatenate([np.stack(p) for p in pairs])
    ctx = api.Context(T)
    _, G, _ = ctx.snr_multi(wins, None, None, _cuda(wA, torch.float64), _cuda(wE, torch.float64),
                            _cuda(th, torch.float64))
    G = G.cpu()
    for w, (rec, inj) in enumerate(pairs):
        rr, ri, ii = G[w, 0, 0], G[w, 0, 1], G[w, 1, 1]
        delta, ov = (rr - 2 * ri + ii) / rr, ri / torch.sqrt(rr * ii)
        od, oo = ogb.match_metrics(wins[w], wA, wE, rec, inj, T)
        assert abs(float(delta - od)) <= 1e-9 * max(1.0, abs(float(od))), (w, float(delta), float(od))
        assert abs(float(ov - oo)) <= 1e-10, (w, float(ov), float(oo))
    ctx.close()
