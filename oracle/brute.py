"""Brute-force time-domain simulation of the same physics, plain FP64 numpy.

TEST INFRASTRUCTURE (see the package docstring).

This module re-derives the detector response without the fast/slow split, so
that the fast/slow oracle in ``gb.py`` can be checked against the physics it
approximates.  It shares no code with ``gb.py``.  At every time sample t = j dt:

* the real strain h_ab(t, x) = Re[H_ab exp(i Phi(t - k.x/c))] is evaluated at
  each event it is needed at;
* one link, emitter i -> receiver j read at time t, takes the emitter at the
  emission time t - L/c and at its position then, and the photon direction
  n = (x_j(t) - x_i(t - L/c)) / |...|:
      y_ij(t) = 1/2 n.[h(t - L/c, x_i(t - L/c)) - h(t, x_j(t))].n / (1 - k.n);
* the first-generation Michelson combination uses exact delays of L/c:
      X(t) = y_21(t) + y_12(t-L) - y_31(t) - y_13(t-L)
             - y_21(t-2L) - y_12(t-3L) + y_31(t-2L) + y_13(t-3L),
  Y and Z cyclically, A = (Z - X)/sqrt2, E = (X - 2Y + Z)/sqrt6 (Eq. 5);
* the spectrum is dt times the DFT of the whole series (continuous-Fourier
  convention), computed with numpy's FFT.

The conventions (orbit, polarisation, link sign, TDI sign) are the readings
R3-R6 listed in ``gb.py``; only their implementation is independent here.
"""
import math

import numpy as np

C_LIGHT = 299792458.0
AU = 1.495978707e11
YEAR = 31557600.0


def _positions(t, L):
    """(3 craft, 3 xyz, len t) positions on the rigid first-order orbit."""
    ecc = L / (2.0 * math.sqrt(3.0) * AU)
    a = 2.0 * np.pi * t / YEAR
    out = np.empty((3, 3, t.size))
    for i in range(3):
        b = 2.0 * np.pi * i / 3.0
        out[i, 0] = AU * (np.cos(a) + 0.5 * ecc * (np.cos(2 * a - b) - 3 * np.cos(b)))
        out[i, 1] = AU * (np.sin(a) + 0.5 * ecc * (np.sin(2 * a - b) - 3 * np.sin(b)))
        out[i, 2] = -math.sqrt(3.0) * AU * ecc * np.cos(a - b)
    return out


def _source(theta):
    f0, fdot, beta, lam, A, iota, psi, phi0 = [float(v) for v in theta]
    khat = -np.array([math.cos(beta) * math.cos(lam), math.cos(beta) * math.sin(lam), math.sin(beta)])
    u = np.array([math.sin(beta) * math.cos(lam), math.sin(beta) * math.sin(lam), -math.cos(beta)])
    v = np.array([math.sin(lam), -math.cos(lam), 0.0])
    ep = np.outer(u, u) - np.outer(v, v)
    ex = np.outer(u, v) + np.outer(v, u)
    Ep = math.cos(2 * psi) * ep - math.sin(2 * psi) * ex
    Ex = math.sin(2 * psi) * ep + math.cos(2 * psi) * ex
    Ap = A * (1.0 + math.cos(iota) ** 2)
    Ax = -2.0 * A * math.cos(iota)
    H = Ap * Ep - 1j * Ax * Ex
    return f0, fdot, phi0, khat, H


def tdi_AE_series(theta, t, L):
    """Real TDI A(t), E(t) at the sample times t (1-D array), exact delays
    (Eq. 5 with the link and Michelson forms of the module docstring)."""
    A, E, _ = tdi_AET_series(theta, t, L)
    return A, E


def tdi_AET_series(theta, t, L):
    """Real TDI A(t), E(t), T(t) = (X + Y + Z)/sqrt3 at the sample times t
    (Eq. 5; T is the third channel of Sec. II, reading R11)."""
    f0, fdot, phi0, khat, H = _source(theta)
    tau = L / C_LIGHT
    # events m = 0..4: time t - m tau, every spacecraft at its position then
    P = [_positions(t - m * tau, L) for m in range(5)]
    phase = []
    for m in range(5):
        xi = (t - m * tau)[None, :] - np.einsum("c,scn->sn", khat, P[m]) / C_LIGHT
        phase.append(2 * np.pi * f0 * xi + np.pi * fdot * xi * xi + phi0)

    def y(i, j, d):
        xr, xe = P[d][j], P[d + 1][i]
        n = xr - xe
        n = n / np.sqrt((n * n).sum(0))
        nHn = np.einsum("an,ab,bn->n", n, H, n)
        kn = khat @ n
        he = (nHn * np.exp(1j * phase[d + 1][i])).real
        hr = (nHn * np.exp(1j * phase[d][j])).real
        return 0.5 * (he - hr) / (1.0 - kn)

    def michelson(c, p, r):
        return (y(p, c, 0) + y(c, p, 1) - y(r, c, 0) - y(c, r, 1)
                - y(p, c, 2) - y(c, p, 3) + y(r, c, 2) + y(c, r, 3))

    X = michelson(0, 1, 2)
    Y = michelson(1, 2, 0)
    Z = michelson(2, 0, 1)
    return (Z - X) / math.sqrt(2.0), (X - 2.0 * Y + Z) / math.sqrt(6.0), (X + Y + Z) / math.sqrt(3.0)


def brute_force_spectrum_aet(theta, T, dt, bins, L=2.5e9, chunk=1 << 16):
    """brute_force_spectrum() with T: (A~, E~, T~) at the given bins (Sec. II, R11)."""
    n_tot = int(round(T / dt))
    out = np.empty((3, n_tot))
    for s in range(0, n_tot, chunk):
        e = min(n_tot, s + chunk)
        t = np.arange(s, e, dtype=np.float64) * dt
        out[:, s:e] = tdi_AET_series(theta, t, L)
    bins = np.asarray(bins)
    return tuple(np.fft.rfft(x)[bins] * dt for x in out)


def brute_force_spectrum(theta, T, dt, bins, L=2.5e9, chunk=1 << 16):
    """dt * DFT of the time-domain A, E series over [0, T), at the given bins
    (the continuous-Fourier convention of the inner product, Eq. 3).

    theta: one parameter vector (8,); bins: integer frequency bins k (f = k/T).
    Returns (A~, E~) complex arrays with len(bins) entries.
    """
    n_tot = int(round(T / dt))
    A = np.empty(n_tot)
    E = np.empty(n_tot)
    for s in range(0, n_tot, chunk):
        e = min(n_tot, s + chunk)
        t = np.arange(s, e, dtype=np.float64) * dt
        A[s:e], E[s:e] = tdi_AE_series(theta, t, L)
    FA = np.fft.rfft(A) * dt
    FE = np.fft.rfft(E) * dt
    bins = np.asarray(bins)
    return FA[bins], FE[bins]
