"""Pins of the paired KDE proposal oracle (Sec. III.G, Alg. 4) against closed
forms, hand examples and sampling statistics."""
import math

import numpy as np
import pytest
from scipy.stats import chi2, norm

from oracle import kde


def test_reduced_box_follows_the_paper():
    mle = np.array([3e-3, 1e-16, 0.2, 1.0, 1e-22, 0.7, 1.0, 2.0])
    sig = np.array([1e-9, 1e-18, 0.01, 0.02, 1e-24, 0.05, 0.1, 0.2])
    plo = np.array([2.9e-3, 0.0, -np.pi / 2, -np.pi, 1e-23, 0.0, 0.0, 0.0])
    phi = np.array([3.1e-3, 5e-16, np.pi / 2, np.pi, 1e-21, 0.72, np.pi, 2 * np.pi])
    lo, hi = kde.reduced_box(mle, sig, plo, phi)
    assert lo[0] == mle[0] - sig[0] and hi[0] == mle[0] + sig[0]          # f0: one sigma
    assert lo[1] == plo[1] and hi[1] == phi[1]                              # fdot: the whole prior
    for d in (2, 3, 4):
        assert lo[d] == pytest.approx(mle[d] - 4 * sig[d]) and hi[d] == pytest.approx(mle[d] + 4 * sig[d])
    assert lo[5] == pytest.approx(mle[5] - 4 * sig[5]) and hi[5] == phi[5]  # cut to the prior
    assert hi[6] - lo[6] == pytest.approx(2 * np.pi / 1000)
    assert hi[7] - lo[7] == pytest.approx(4 * np.pi / 1000)


def test_accepted_moves_hand_example():
    assert kde.accepted_moves([0, 0, 2, 2, 4]) == 2
    assert kde.accepted_moves([0]) == 0
    assert kde.accepted_moves([0, 1, 2, 3]) == 3


def test_flat_grid_is_uniform_in_the_box():
    G = 16
    C = np.stack([kde.cumulative(kde.flat_grid(G))] * 3)
    lo = np.array([1.0, -2.0, 0.1, 0.3, 5.0, 0.0, 0.5, 1.0])
    hi = np.array([1.5, 2.0, 0.4, 0.9, 6.0, 0.2, 0.6, 1.3])
    vol = float(np.prod(hi - lo))
    rng = np.random.default_rng(3)
    pts = []
    for _ in range(4000):
        th, lg, lu = kde.draw(C, kde.box_extents(lo, hi), lo, hi, G, rng.integers(0, 2 ** 32, 12))
        assert lg == pytest.approx(-math.log(vol), rel=1e-12)
        assert lu < 0
        pts.append(th)
    pts = (np.array(pts) - lo) / (hi - lo)
    assert pts.min() >= 0 and pts.max() < 1
    # each coordinate uniform on [0, 1): mean 1/2, variance 1/12
    assert np.allclose(pts.mean(0), 0.5, atol=0.02) and np.allclose(pts.var(0), 1 / 12, atol=0.01)


def test_single_state_puts_the_kde_mass_in_its_cell():
    # zero spread: no smoothing, a grid of one box cell either side of the
    # state (the state in its middle cell), every entry in that cell, plus the floor
    G, eps = 7, 0.05
    x, y = np.full(50, 0.33), np.full(50, 0.71)
    P, (ex, ey) = kde.pair_grid(x, y, 1, (0.0, 1.0), (0.0, 2.0), G, eps)
    assert ex == pytest.approx((0.33 - 1 / 7, 0.33 + 1 / 7)) and ey == pytest.approx((0.71 - 2 / 7, 0.71 + 2 / 7))
    expect = np.full((G, G), eps / G ** 2)
    expect[3, 3] += 1 - eps
    assert np.allclose(P, expect, rtol=0, atol=1e-15)
    # at the box edge the grid is cut to the box
    _, (ex, _) = kde.pair_grid(np.full(5, 0.01), np.full(5, 0.5), 1, (0.0, 1.0), (0.0, 1.0), G, eps)
    assert ex == pytest.approx((0.0, 0.01 + 1 / 7))


def test_kernel_smoothing_of_one_entry_is_the_discrete_gaussian():
    # one entry in the middle of a 33 x 33 grid, axis bandwidths 2 and 3 cells
    G = 33
    k2, r2 = kde.kernel_weights(2.0, G)
    k3, r3 = kde.kernel_weights(3.0, G)
    assert r2 == 6 and r3 == 9
    d = np.arange(-6, 7)
    assert np.allclose(k2, np.exp(-d ** 2 / 8) / np.exp(-d ** 2 / 8).sum())
    H = np.zeros((G, G))
    H[16, 16] = 1
    S = kde.smoothing_matrix(2.0, G) @ H @ kde.smoothing_matrix(3.0, G).T
    assert np.allclose(S[10:23, 16], k2 * k3[9]) and np.allclose(S[16, 7:26], k2[6] * k3)
    assert S.sum() == pytest.approx(1.0)


def test_grid_of_a_gaussian_sample_matches_the_smoothed_gaussian():
    # independent normals in x and y with different widths: the estimate is,
    # up to sampling noise and cell discretisation, the normal of variance
    # s^2 + h^2 per axis integrated over the cells (a transposed kernel or a
    # wrong bandwidth fails the total-variation bound)
    rng = np.random.default_rng(11)
    n, G = 200000, 48
    x = rng.normal(0.2, 0.05, n)
    y = rng.normal(-0.1, 0.2, n)
    bx, by = (0.0, 0.4), (-0.9, 0.7)
    P, (gx, gy) = kde.pair_grid(x, y, n, bx, by, G, 0.0)
    h = n ** (-1 / 6)
    # the grid spans the sample's range +- 3h (and a box cell), inside the box
    assert gx[0] == pytest.approx(max(bx[0], x.min() - 3 * 0.05 * h - 0.4 / G), rel=1e-6)
    assert gy[1] == pytest.approx(min(by[1], y.max() + 3 * 0.2 * h + 1.6 / G), rel=1e-6)
    ex = np.linspace(gx[0], gx[1], G + 1)
    ey = np.linspace(gy[0], gy[1], G + 1)
    cx, cy = (gx[1] - gx[0]) / G, (gy[1] - gy[0]) / G
    # histogram binning adds a cell^2/12 variance, the discrete kernel its own
    sx = math.sqrt(0.05 ** 2 * (1 + h ** 2) + cx ** 2 / 12)
    sy = math.sqrt(0.2 ** 2 * (1 + h ** 2) + cy ** 2 / 12)
    qx = np.diff(norm.cdf(ex, 0.2, sx))
    qy = np.diff(norm.cdf(ey, -0.1, sy))
    Q = np.outer(qx, qy)
    Q /= Q.sum()
    # sampling noise alone gives about 0.010 here (the noise-free estimate is
    # within 0.001 of Q); the bound fails for swapped axis bandwidths (0.054),
    # no smoothing (0.028) or twice the bandwidth (0.017)
    assert 0.5 * np.abs(P - Q).sum() < 0.0125
    H = np.histogram2d(x, y, bins=[ex, ey])[0]
    for fx, fy in ((0.2 / 0.05, 0.05 / 0.2), (2.0, 2.0)):
        Pw = kde.smoothing_matrix(fx * 0.05 * h / cx, G) @ H @ kde.smoothing_matrix(fy * 0.2 * h / cy, G).T
        Pw /= Pw.sum()
        assert 0.5 * np.abs(Pw - Q).sum() > 0.015


def test_draws_follow_the_cell_probabilities():
    G = 8
    rng = np.random.default_rng(5)
    P = rng.gamma(1.0, size=(G, G))
    P /= P.sum()
    C = np.stack([kde.cumulative(P), kde.cumulative(kde.flat_grid(G)), kde.cumulative(kde.flat_grid(G))])
    lo, hi = np.zeros(8), np.ones(8)
    hi[0], hi[1] = 2.0, 4.0
    counts = np.zeros(G * G)
    m = 40000
    for _ in range(m):
        th, lg, _ = kde.draw(C, kde.box_extents(lo, hi), lo, hi, G, rng.integers(0, 2 ** 32, 12))
        i, j = int(th[0] / 2.0 * G), int(th[1] / 4.0 * G)
        counts[i * G + j] += 1
        # log g: the drawn cell's probability over its area, the rest flat
        assert lg == pytest.approx(math.log(P[i, j] / (2.0 / G * 4.0 / G)), rel=1e-9, abs=1e-9)
    expect = m * P.ravel()
    stat = float(((counts - expect) ** 2 / expect).sum())
    assert stat < chi2.ppf(0.999, G * G - 1)


def test_build_window_uses_the_chain_states():
    # the estimate sees the chain's states with their step counts, not the proposals
    rng = np.random.default_rng(2)
    n, G = 400, 16
    theta = rng.uniform(0.0, 1.0, (n, 8))
    chain = np.zeros(n, int)
    chain[200:] = 200                     # two states: proposal 0, then 200
    lo, hi = np.zeros(8), np.ones(8)
    C, E = kde.build_window(theta, chain, lo, hi, G, 0.0)
    for p, (dx, dy) in enumerate(kde.PAIRS):
        P = np.diff(np.concatenate([[0.0], C[p]])).reshape(G, G)
        x0, x1, y0, y1 = E[p]
        assert x0 <= min(theta[0, dx], theta[200, dx]) and x1 >= max(theta[0, dx], theta[200, dx])
        a = (kde.cell_index(theta[0, dx], x0, x1, G), kde.cell_index(theta[0, dy], y0, y1, G))
        b = (kde.cell_index(theta[200, dx], x0, x1, G), kde.cell_index(theta[200, dy], y0, y1, G))
        if a != b:
            assert P[a] == pytest.approx(P[b], rel=1e-9)     # 200 steps each
        assert P.sum() == pytest.approx(1.0)


def test_product_reduced_box_matches_the_oracle():
    # the driver's host-side reduced box (no GPU needed) against the oracle's
    from paper_2307_03763_gb300.posterior import reduced_box
    rng = np.random.default_rng(8)
    plo = np.array([2.9e-3, 0.0, -np.pi / 2, -np.pi, 1e-24, 0.0, 0.0, 0.0])
    phi = np.array([3.1e-3, 5e-16, np.pi / 2, np.pi, 1e-20, np.pi, np.pi, 2 * np.pi])
    mle = plo + (phi - plo) * rng.uniform(size=(20, 8))
    sig = (phi - plo) * rng.uniform(0.001, 0.3, size=(20, 8))
    got = reduced_box(mle, sig, plo, phi)
    for w in range(20):
        lo, hi = kde.reduced_box(mle[w], sig[w], plo, phi)
        assert np.array_equal(got[w, :8], lo) and np.array_equal(got[w, 8:], hi)
