"""gb_noise_median against the oracle's median periodogram (Sec. III.C):
exact per window (a median of the same doubles), odd and even W, a window
with loud signals, W = 0, and the weights it writes."""
import math

import numpy as np
import pytest
import torch

from oracle import noise as onoise
from paper_2307_03763_gb300 import workloads as wk

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def api():
    from paper_2307_03763_gb300 import api, build
    build.build()
    return api


@pytest.mark.parametrize("debias", [False, True])
def test_noise_median_matches_oracle(api, debias):
    T = 2 * wk.YEAR
    ctx = api.Context(T)
    rng = np.random.default_rng(12)
    Ws = [128, 1000, 1, 4096, 0, 257, 64]
    offs = np.cumsum([0] + Ws)
    nb = int(offs[-1])
    S0 = 10 ** rng.uniform(-42, -39, len(Ws))
    d = np.empty((2, nb), np.complex128)
    for c in range(2):
        for w, W in enumerate(Ws):
            s = math.sqrt(T * S0[w] * (1 + c) / 4)
            d[c, offs[w]:offs[w] + W] = rng.normal(0, s, W) + 1j * rng.normal(0, s, W)
    d[0, offs[1] + 10:offs[1] + 13] *= 1e4                         # loud bins in window 1
    wins = [(int(1000 * w), W, 128, int(offs[w]), 0, 0) for w, W in enumerate(Ws)]
    dA, dE = (torch.as_tensor(d[c], device=DEV) for c in range(2))
    wA = torch.zeros(nb, dtype=torch.float64, device=DEV)
    wE = torch.zeros(nb, dtype=torch.float64, device=DEV)
    S = ctx.noise_median(wins, dA, dE, debias=debias, weights=(wA, wE)).cpu().numpy()
    wA, wE = wA.cpu().numpy(), wE.cpu().numpy()
    for w, W in enumerate(Ws):
        if W == 0:
            assert np.isnan(S[w]).all()
            continue
        for c, wt in ((0, wA), (1, wE)):
            ref = onoise.median_psd(d[c, offs[w]:offs[w] + W], T, debias=debias)
            assert S[w, c] == ref, (w, c, S[w, c], ref)
            assert np.all(wt[offs[w]:offs[w] + W] == 1.0 / ref)
    # with 1,000 bins the debiased estimate is the injected PSD within a few percent
    if debias:
        assert S[1, 0] == pytest.approx(S0[1], rel=0.15) and S[3, 1] == pytest.approx(2 * S0[3], rel=0.1)
