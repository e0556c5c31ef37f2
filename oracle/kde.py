"""Paired two-dimensional kernel-density proposals of the annealed posterior, plain FP64.

TEST INFRASTRUCTURE (see the package docstring).

Sec. III.G: the posterior of one recovered signal is sampled by the
independence Metropolis-Hastings chain of Alg. 4 over a reduced parameter
space around the MLE.  The first temperature draws uniformly from that space;
afterwards the posterior obtained at one temperature, smoothed by a kernel
density estimate, is the proposal of the next.  To keep the estimates
two-dimensional the parameters are grouped in pairs, A-iota, lambda-beta and
f-fdot, with one estimate per pair; polarisation and initial phase are not
estimated (their range is narrow).  The paper names the KDE technique only by
citation; the readings below fix a grid estimate that can be both sampled and
evaluated exactly.

Readings
--------
K1  Pairs (theta indices): (f0, fdot) = (0, 1), (lambda, beta) = (3, 2),
    (A, iota) = (4, 5).  psi (6) and phi0 (7) are uniform over their reduced
    ranges at every temperature.  The proposal density is the product of the
    three pair densities and the two uniform ones.
K2  Reduced space (the box of Sec. III.G): theta_MLE +- 4 sigma, f0 +- sigma_f,
    fdot over its whole prior range, psi +- pi/1000, phi0 +- 2 pi/1000, every
    range cut to the prior box; sigma = sqrt(diag F^-1).
K3  Grid estimate of one pair.  The grid spans the chain's own range on each
    axis, as kernel-density grids do: [max(lo, a - 3h - c0), min(hi,
    b + 3h + c0)] for entries in [a, b], bandwidth h and the box cell
    c0 = (hi - lo)/G, so that its resolution follows the posterior (fdot's
    reduced range is its whole prior, thousands of posterior widths at high
    frequency); the first temperature's grids span the box.  On that extent
    [lo', hi'] with G x G cells (cell (i, j) covers x in lo' + [i, i+1) c,
    c = (hi' - lo')/G, and likewise y):
      * the chain's n entries (each step counts the state it is in, so a
        state weighs the steps spent in it) are counted per cell, cell index
        floor((x - lo') / (hi' - lo') * G) clamped to [0, G-1];
      * the counts are smoothed by a Gaussian kernel per axis with Scott's
        bandwidth for two dimensions, h = s n_eff^(-1/6), s the standard
        deviation of the n entries (divisor n) and n_eff the number of
        distinct visits, accepted moves + 1; in cells sigma = h / c, the
        weights exp(-d^2 / (2 sigma^2)) for |d| <= r = min(ceil(3 sigma), G-1)
        normalised to sum one (sigma = 0: no smoothing); mass pushed past the
        grid edge is dropped;
      * the result is normalised to one and mixed with a uniform floor:
        P = (1 - eps) S / sum S + eps / G^2, so every cell keeps a chance.
K4  The density is constant on a cell of the pair's grid.  A draw picks
    cell c (flattened c = i G + j) with probability P_c through the
    cumulative sums
    C_c = P_0 + ... + P_c: the first c with C_c > u (the last cell if none),
    then a uniform point in it.  P_c is taken as C_c - C_(c-1) (C_(-1) = 0),
    the probability the draw actually has, and
    log g = sum_pairs log(P_c / (c_x c_y)) - log(width psi) - log(width phi0).
K5  The first temperature uses flat grids over the box, P_c = 1/G^2:
    uniform in the box.
K6  Between temperatures the estimate is used as it is, without rescaling
    for the next temperature (the paper uses the obtained posterior as the
    next proposal).
K7  Random numbers are inputs: twelve 32-bit words per proposal, u = (w + 1/2)
    2^-32; words 3p, 3p+1, 3p+2 give pair p's cell, x and y; word 9 psi,
    word 10 phi0, word 11 the log u of the chain.
"""
import math

import numpy as np

PAIRS = ((0, 1), (3, 2), (4, 5))


def reduced_box(mle, sigma, prior_lo, prior_hi):
    """The reduced parameter space of Sec. III.G (reading K2); arrays of 8."""
    mle, sigma = np.asarray(mle, float), np.asarray(sigma, float)
    prior_lo, prior_hi = np.asarray(prior_lo, float), np.asarray(prior_hi, float)
    half = 4.0 * sigma
    half[0] = sigma[0]
    lo, hi = mle - half, mle + half
    lo[1], hi[1] = prior_lo[1], prior_hi[1]
    lo[6], hi[6] = mle[6] - math.pi / 1000, mle[6] + math.pi / 1000
    lo[7], hi[7] = mle[7] - 2 * math.pi / 1000, mle[7] + 2 * math.pi / 1000
    for d in range(6):   # psi and phi0 are periodic: their narrow range stays as it is
        lo[d], hi[d] = max(lo[d], prior_lo[d]), min(hi[d], prior_hi[d])
    return lo, hi


def accepted_moves(chain):
    """Number of i >= 1 where the chain moved to proposal i (the acceptances of Alg. 4)."""
    return sum(1 for i in range(1, len(chain)) if chain[i] == i)


def kernel_weights(sigma, G):
    """Truncated, normalised Gaussian weights for offsets -r..r (reading K3)."""
    if not (sigma > 0.0) or not math.isfinite(sigma):
        return np.array([1.0]), 0
    r = min(int(math.ceil(3.0 * sigma)), G - 1)
    d = np.arange(-r, r + 1, dtype=float)
    k = np.exp(-d * d / (2.0 * sigma * sigma))
    return k / k.sum(), r


def smoothing_matrix(sigma, G):
    """G x G matrix M with (M v)_i = sum_d k_d v_(i-d), zero outside the grid
    (the Gaussian smoothing of reading K3)."""
    k, r = kernel_weights(sigma, G)
    M = np.zeros((G, G))
    for i in range(G):
        for d in range(-r, r + 1):
            if 0 <= i - d < G:
                M[i, i - d] = k[d + r]
    return M


def cell_index(v, lo, hi, G):
    """Grid cell of v on [lo, hi) with G cells, clamped to the grid (reading K3)."""
    i = math.floor((v - lo) / (hi - lo) * G)
    return min(max(i, 0), G - 1)


def grid_extent(v, h, lo, hi, G):
    """[lo', hi'] of one axis (reading K3)."""
    c0 = (hi - lo) / G
    return max(lo, float(np.min(v)) - 3.0 * h - c0), min(hi, float(np.max(v)) + 3.0 * h + c0)


def pair_grid(x, y, n_eff, box_x, box_y, G, eps):
    """Cell probabilities P (G x G, x index first) of one pair and the grid's
    extents ((lo'_x, hi'_x), (lo'_y, hi'_y)) (reading K3).

    x, y: the n chain entries of the pair's two parameters."""
    x, y = np.asarray(x, float), np.asarray(y, float)
    n = len(x)
    bw = n_eff ** (-1.0 / 6.0)
    hx, hy = x.std() * bw, y.std() * bw
    ex, ey = grid_extent(x, hx, box_x[0], box_x[1], G), grid_extent(y, hy, box_y[0], box_y[1], G)
    H = np.zeros((G, G))
    for a, b in zip(x, y):
        H[cell_index(a, ex[0], ex[1], G), cell_index(b, ey[0], ey[1], G)] += 1.0
    cx, cy = (ex[1] - ex[0]) / G, (ey[1] - ey[0]) / G
    S = smoothing_matrix(hx / cx, G) @ H @ smoothing_matrix(hy / cy, G).T
    assert n > 0 and S.sum() > 0
    return (1.0 - eps) * S / S.sum() + eps / (G * G), (ex, ey)


def flat_grid(G):
    """The uniform first-temperature density over the box (reading K5)."""
    return np.full((G, G), 1.0 / (G * G))


def cumulative(P):
    """C_c over the flattened cells c = i G + j (reading K4)."""
    return np.cumsum(np.asarray(P, float).ravel())


def build_window(theta, chain, lo, hi, G, eps):
    """Cumulative sums of the three pair grids of one window from its chain
    (readings K1, K3, K4; Sec. III.G),
    and their extents: theta (n, 8) proposals, chain (n) state index after
    each step.  Returns (C (3, G^2), E (3, 4) = lo'_x, hi'_x, lo'_y, hi'_y)."""
    theta = np.asarray(theta, float)
    states = theta[np.asarray(chain, int)]
    n_eff = accepted_moves(chain) + 1
    C, E = [], []
    for dx, dy in PAIRS:
        P, (ex, ey) = pair_grid(states[:, dx], states[:, dy], n_eff, (lo[dx], hi[dx]), (lo[dy], hi[dy]), G, eps)
        C.append(cumulative(P))
        E.append([ex[0], ex[1], ey[0], ey[1]])
    return np.stack(C), np.array(E)


def box_extents(lo, hi):
    """The pairs' extents of the first temperature: the box (reading K5)."""
    return np.array([[lo[dx], hi[dx], lo[dy], hi[dy]] for dx, dy in PAIRS])


def u01(word):
    """A 32-bit Philox word as a uniform variate in (0, 1): (word + 1/2) / 2^32 (reading K7)."""
    return (int(word) + 0.5) * 2.0 ** -32


def draw(cdfs, exts, lo, hi, G, words):
    """One proposal from the three pairs' cumulative sums over their extents
    (reading K4, K7); lo, hi: the box (psi and phi0).

    Returns (theta[8], log_g, log_u)."""
    theta = np.zeros(8)
    log_g = 0.0
    for p, (dx, dy) in enumerate(PAIRS):
        C = cdfs[p]
        u = u01(words[3 * p])
        c = 0
        while c < G * G - 1 and C[c] <= u:
            c += 1
        Pc = C[c] - (C[c - 1] if c > 0 else 0.0)
        i, j = divmod(c, G)
        x0, x1, y0, y1 = exts[p]
        cx, cy = (x1 - x0) / G, (y1 - y0) / G
        theta[dx] = x0 + (i + u01(words[3 * p + 1])) * cx
        theta[dy] = y0 + (j + u01(words[3 * p + 2])) * cy
        log_g += math.log(Pc) - math.log(cx * cy)
    for d, w in ((6, 9), (7, 10)):
        theta[d] = lo[d] + u01(words[w]) * (hi[d] - lo[d])
        log_g -= math.log(hi[d] - lo[d])
    return theta, log_g, math.log(u01(words[11]))
