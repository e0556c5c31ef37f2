"""Test-side helpers: build data windows by injecting oracle templates into noise.

Tests may call the oracle; the product path never does.  Every array produced
here comes from the seeded generators in ``paper_2307_03763_gb300.workloads``
plus the oracle's own template, never from the CUDA path.
"""
import numpy as np
import torch

from oracle import gb as ogb


def template_on_window(src, k0, W, N, T):
    """Oracle template of one source restricted to window bins [k0, k0+W)."""
    q, hA, hE = ogb.template(torch.tensor(np.asarray(src)[None, :]), N, T)
    q = int(q[0])
    outA = np.zeros(W, np.complex128)
    outE = np.zeros(W, np.complex128)
    j = q - N // 2 + np.arange(N) - k0
    ok = (j >= 0) & (j < W)
    outA[j[ok]] = hA[0].numpy()[ok]
    outE[j[ok]] = hE[0].numpy()[ok]
    return outA, outE


def inject(wl, sources=None):
    """Data = noise + sum of the oracle templates of each window's sources."""
    dA = wl.noise_A.copy()
    dE = wl.noise_E.copy()
    srcs = wl.sources if sources is None else sources
    for w, (k0, W, N, doff, coff, nc) in enumerate(wl.windows):
        for s in srcs[w]:
            hA, hE = template_on_window(s, k0, W, N, wl.T)
            dA[doff:doff + W] += hA
            dE[doff:doff + W] += hE
    return dA, dE


def unit_snr(src, window, wA, wE, T):
    """<h|h>^(1/2) of a source on its window (oracle), for rescaling A to a target SNR."""
    k0, W, N, doff, _, _ = window
    hA, hE = template_on_window(src, k0, W, N, T)
    hh = (4.0 / T) * (np.sum(wA[doff:doff + W] * np.abs(hA) ** 2) + np.sum(wE[doff:doff + W] * np.abs(hE) ** 2))
    return float(np.sqrt(hh))


def fisher_matrix(src, window, wA, wE, T, rel=1e-4):
    """F_ij = <d_i h|d_j h> on the window (oracle templates, central differences)."""
    k0, W, N, doff, _, _ = window
    wa, we = wA[doff:doff + W], wE[doff:doff + W]
    scales = np.array([1.0 / T, 1.0 / T ** 2, 1.0, 1.0, src[4], 1.0, 1.0, 1.0])
    J = []
    for i in range(8):
        h = rel * scales[i]
        tp, tm = src.copy(), src.copy()
        tp[i] += h
        tm[i] -= h
        ap, ep = template_on_window(tp, k0, W, N, T)
        am, em = template_on_window(tm, k0, W, N, T)
        J.append(((ap - am) / (2 * h), (ep - em) / (2 * h)))
    F = np.empty((8, 8))
    for i in range(8):
        for j in range(8):
            F[i, j] = (4.0 / T) * (np.sum(wa * (J[i][0] * J[j][0].conj()).real)
                                   + np.sum(we * (J[i][1] * J[j][1].conj()).real))
    return F


def fisher_sigma(src, window, wA, wE, T, rel=1e-4):
    """sqrt(diag F^-1) of the window's Fisher matrix, inverted in natural units
    (1/T, 1/T^2, rad, A): in SI units its entries span ~70 decades, beyond the
    reach of a pseudo-inverse's relative cut-off."""
    F = fisher_matrix(src, window, wA, wE, T, rel)
    sc = np.array([1.0 / T, 1.0 / T ** 2, 1.0, 1.0, src[4], 1.0, 1.0, 1.0])
    return np.sqrt(np.abs(np.diag(np.linalg.pinv(F * np.outer(sc, sc))))) * sc
