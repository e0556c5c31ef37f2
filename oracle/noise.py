"""Noise estimate within a frequency segment, plain FP64.

TEST INFRASTRUCTURE (see the package docstring).

Sec. III.C: the noise of each segment is estimated from the periodogram of
its (padded) window, S(f) = 2 |A(f)|^2 / (N f_sample), and the median over
the window is taken as a constant estimate for the whole segment, so that
loud signals inside it barely move it.  It is updated after every subtracted
signal, and E (and T) are estimated alike.

Readings
--------
N1  The data here are continuous-Fourier-transform samples d(f_k) = dt DFT_k
    (the convention of the likelihood), so the paper's 2 |DFT|^2 / (N f_s)
    with N the number of time samples is 2 |d(f_k)|^2 / T.  (The paper calls
    N the number of bins of the padded window, which does not give a PSD.)
N2  The median is that of the W window bins (for even W the mean of the two
    middle values); the value is 2 (Re^2 + Im^2) / T per bin in that order.
N3  For Gaussian noise |d|^2 is exponential, whose median is ln 2 times its
    mean: the median as printed is S ln 2.  debias=True divides by ln 2 for
    an unbiased estimate; the default is the literal median.
"""
import math

import numpy as np

LN2 = math.log(2.0)


def periodogram(d, T):
    """2 |d_k|^2 / T per bin (readings N1, N2)."""
    d = np.asarray(d, dtype=np.complex128)
    return 2.0 * (d.real * d.real + d.imag * d.imag) / T


def median_psd(d, T, debias=False):
    """The segment's constant noise estimate (Sec. III.C; N3)."""
    s = float(np.median(periodogram(d, T)))
    return s / LN2 if debias else s
