"""Pins of the Metropolis-Hastings chain oracle (Alg. 4, Eq. 13)."""
import itertools
import math
import os

import numpy as np
import pytest

from oracle import mh


def _golden(name):
    path = os.path.join(os.path.dirname(__file__), "golden", name)
    out = {}
    for line in open(path):
        line = line.strip()
        if line and not line.startswith("#") and "=" in line:
            k, v = line.split("=")
            out[k] = [float(x) for x in v.split(",")]
    return out


def test_hand_worked_example():
    g = _golden("mh_alg4_worked.txt")
    chain, acc = mh.mh_independence(g["logL"], g["log_g"], g["log_u"], g["temperature"][0])
    assert chain == [int(x) for x in g["chain"]]
    assert acc == int(g["n_accept"][0])


@pytest.mark.parametrize("n", [1, 2, 7])
def test_every_accept_pattern_is_reproduced(n):
    # strictly decreasing logL makes every alpha < 1, so each step can be
    # steered either way by its log u; enumerate all 2^(n-1) patterns
    logL = [-float(i) for i in range(n)]
    log_g = [0.0] * n
    for pattern in itertools.product([False, True], repeat=n - 1):
        c, expect, log_u = 0, [0], [-0.5]
        for i, acc in enumerate(pattern, start=1):
            delta = logL[i] - logL[c]           # < 0
            log_u.append(delta - 0.25 if acc else delta + 0.25)
            if acc:
                c = i
            expect.append(c)
        chain, na = mh.mh_independence(logL, log_g, log_u, 1.0)
        assert chain == expect
        assert na == sum(pattern)


def test_flat_target_accepts_every_move():
    n = 50
    rng = np.random.default_rng(0)
    chain, na = mh.mh_independence([0.0] * n, [0.0] * n, np.log(rng.uniform(1e-300, 1, n)), 3.0)
    assert chain == list(range(n)) and na == n - 1


def test_minus_infinity_is_never_accepted():
    chain, na = mh.mh_independence([0.0, -math.inf, -math.inf, -1.0], [0.0] * 4, [-1e-9, -1e-9, -1e-9, -2.0], 1.0)
    assert chain == [0, 0, 0, 3]
    chain, na = mh.mh_independence([-math.inf, -math.inf, 2.0], [0.0] * 3, [-1e-9] * 3, 1.0)
    assert chain == [0, 0, 2]


def test_readings_agree_at_unit_temperature():
    rng = np.random.default_rng(1)
    n = 500
    l, g, u = rng.normal(0, 3, n), rng.normal(0, 1, n), np.log(rng.uniform(0, 1, n))
    assert mh.mh_independence(l, g, u, 1.0) == mh.mh_independence(l, g, u, 1.0, literal=True)


@pytest.mark.parametrize("temperature,var", [(1.0, 1.0), (4.0, 4.0)])
def test_chain_samples_the_tempered_gaussian(temperature, var):
    # target L(x) = N(0,1) so L^(1/T) = N(0, T); independence proposals
    # N(0, 3^2 T) with their exact log density.  The chain mean and variance
    # must match the tempered target within Monte-Carlo error (reading M1).
    rng = np.random.default_rng(2)
    n = 200000
    s = 3.0 * math.sqrt(temperature)
    x = rng.normal(0, s, n)
    logL = -0.5 * x * x
    log_g = -0.5 * (x / s) ** 2
    log_u = np.log(rng.uniform(0, 1, n))
    chain, na = mh.mh_independence(logL, log_g, log_u, temperature)
    xs = x[np.array(chain)]
    ess = n * na / n / 4            # crude effective sample size
    assert abs(xs.mean()) < 5 * math.sqrt(var / ess)
    assert abs(xs.var() - var) < 5 * var * math.sqrt(2 / ess)
