"""Host logic of the synthetic inputs: the analytic noise PSDs, the chirp
scaling of Eq. 8, the Alg. 1 segments and the full-band window layout."""
import math

import numpy as np

from paper_2307_03763_gb300 import workloads as wk


def _single_link_noises(f):
    # acceleration and optical-metrology noise per link, fractional frequency
    s_acc = (3e-15) ** 2 * (1 + (0.4e-3 / f) ** 2) * (1 + (f / 8e-3) ** 4) / (2 * np.pi * f * wk.C_LIGHT) ** 2
    s_oms = (15e-12) ** 2 * (1 + (2e-3 / f) ** 4) * (2 * np.pi * f / wk.C_LIGHT) ** 2
    return s_acc, s_oms


def test_psds_are_the_orthogonal_combinations_of_the_michelson_correlations():
    # first-generation Michelson X with equal arms: auto- and cross-spectra
    #   S_XX = 16 sin^2 x [S_oms + (3 + cos 2x) S_acc]
    #   S_XY = -8 sin^2 x cos x [S_oms + 4 S_acc]
    # A = (Z - X)/sqrt2, E = (X - 2Y + Z)/sqrt6 and T = (X + Y + Z)/sqrt3 are
    # uncorrelated, with S_A = S_E = S_XX - S_XY and S_T = S_XX + 2 S_XY
    f = np.geomspace(1e-4, 1e-1, 400)
    x = 2 * np.pi * f * wk.ARM_L / wk.C_LIGHT
    s_acc, s_oms = _single_link_noises(f)
    sxx = 16 * np.sin(x) ** 2 * (s_oms + (3 + np.cos(2 * x)) * s_acc)
    sxy = -8 * np.sin(x) ** 2 * np.cos(x) * (s_oms + 4 * s_acc)
    assert np.allclose(wk.psd_AE(f), sxx - sxy, rtol=1e-12, atol=0)
    # S_XX + 2 S_XY cancels to S_T << S_XX at low frequency: compare on the
    # scale of the terms
    assert np.all(np.abs(wk.psd_T(f) - (sxx + 2 * sxy)) <= 1e-13 * sxx)
    # at low frequency the T noise is far below the A noise: S_T / S_A -> 0
    assert wk.psd_T(1e-4) / wk.psd_AE(1e-4) < 1e-6


def test_psd_calibration_value():
    # the workloads' calibration point: S_A(1.5 mHz) ~ 8.5e-43 / Hz
    assert abs(wk.psd_AE(1.5e-3) / 8.5e-43 - 1) < 0.01


def test_chirp_fdot_scalings():
    # Eq. 8: fdot ~ Mc^(5/3) f^(11/3)
    f = np.array([1e-3, 3e-3, 1e-2])
    assert np.allclose(wk.chirp_fdot(2 * f, 0.5) / wk.chirp_fdot(f, 0.5), 2 ** (11 / 3), rtol=1e-13)
    assert np.allclose(wk.chirp_fdot(f, 1.0) / wk.chirp_fdot(f, 0.5), 2 ** (5 / 3), rtol=1e-13)
    assert np.all(wk.chirp_fdot(f, 0.5) > 0)


def test_segments_tile_the_band():
    # Alg. 1: contiguous segments [f, f + 2 B_max(f)) from f_min past f_max
    T = 2 * wk.YEAR
    seg = wk.segments(0.3e-3, 15e-3, T)
    assert seg[0][0] == 0.3e-3 and seg[-1][1] >= 15e-3 and seg[-2][1] < 15e-3
    for (a, b), (c, _) in zip(seg[:-1], seg[1:]):
        assert b == c
    for a, b in seg:
        assert math.isclose(b - a, 2 * float(wk.bandwidth_max(a, T)), rel_tol=1e-12)
    # B_max = B_F + 2 B_O + 2 B_C: at least the two 4/yr Doppler terms
    assert all(b - a >= 16.0 / wk.YEAR for a, b in seg)


def test_fullband_layout_windows_hold_their_segments():
    T = 2 * wk.YEAR
    lay = wk.fullband_layout(0.3e-3, 15e-3, T, n_cap=1024)
    prev_kb = None
    for k0, N, ka, kb in lay:
        assert N & (N - 1) == 0 and 32 <= N <= 1024
        assert kb - ka <= N and N < 2 * max(kb - ka, 16)     # the smallest power of two that holds it
        assert k0 <= ka and kb <= k0 + N                      # the window covers its segment
        if prev_kb is not None:
            assert prev_kb - 1 <= ka <= prev_kb               # consecutive segments share at most one bin
        prev_kb = kb
    assert lay[0][2] == math.floor(0.3e-3 * T)
    # a cap smaller than the widest segment splits it into equal parts
    small = wk.fullband_layout(10e-3, 11e-3, T, n_cap=128)
    assert all(N <= 128 for _, N, _, _ in small)
    assert len(small) > len(wk.fullband_layout(10e-3, 11e-3, T, n_cap=1024))


def test_n_for_band_is_the_smallest_power_of_two():
    T = wk.YEAR
    for f in (0.5e-3, 2e-3, 6e-3, 12e-3, 19e-3):
        n = wk.n_for_band(f, T)
        bins = 2 * float(wk.bandwidth_max(f, T, 1.0)) * T
        assert n & (n - 1) == 0 and n >= 32 and n >= bins and (n == 32 or n / 2 < bins)
