"""Pins of the segment noise estimate (Sec. III.C) against statistics of
simulated noise with a known PSD, its robustness to loud bins, and the
closed form of one bin."""
import math

import numpy as np
import pytest

from oracle import noise


def test_periodogram_of_one_bin():
    T = 1e7
    assert noise.periodogram([3.0 + 4.0j], T)[0] == pytest.approx(2 * 25 / T, rel=1e-15)


def test_median_of_gaussian_noise_is_ln2_times_the_psd():
    # Re, Im ~ N(0, T S / 4) (the one-sided PSD S in the continuous-FT convention)
    rng = np.random.default_rng(4)
    T, S, n = 6.3e7, 3.7e-41, 200001
    d = rng.normal(0, math.sqrt(T * S / 4), n) + 1j * rng.normal(0, math.sqrt(T * S / 4), n)
    assert noise.periodogram(d, T).mean() == pytest.approx(S, rel=0.01)
    assert noise.median_psd(d, T) == pytest.approx(S * math.log(2), rel=0.01)
    assert noise.median_psd(d, T, debias=True) == pytest.approx(S, rel=0.01)


def test_median_ignores_a_few_loud_bins():
    rng = np.random.default_rng(5)
    T, S, n = 3.15e7, 1e-40, 1000
    d = rng.normal(0, math.sqrt(T * S / 4), n) + 1j * rng.normal(0, math.sqrt(T * S / 4), n)
    loud = d.copy()
    loud[400:404] *= 1e3
    assert noise.median_psd(loud, T) == pytest.approx(noise.median_psd(d, T), rel=0.01)
    assert noise.periodogram(loud, T).mean() > 100 * noise.periodogram(d, T).mean()


def test_even_count_median_is_the_mean_of_the_middle_pair():
    T = 2.0
    d = np.sqrt(np.array([1.0, 4.0, 2.0, 3.0]))
    assert noise.median_psd(d, T) == 2.5
