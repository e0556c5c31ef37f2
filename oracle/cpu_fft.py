"""A second CPU timing baseline: the oracle's likelihood with a radix-2 FFT.

TEST INFRASTRUCTURE (see the package docstring).  This module is not one of
the oracle's checked functions: it exists so that the CPU throughput that
bench.py reports beside the GPU is not only that of the naive O(N^2) DFT.
Every step is the oracle's (gb.slow_part for R1-R7, gb.window_inner_products
for R9-R10) except the transform of R8, which here is an iterative radix-2
decimation-in-time FFT written for this purpose (bit-reversed input, log2 N
butterfly stages, vectorised over the candidates).  Its agreement with the
oracle's DFT is checked in tests/test_oracle_pins.py.
"""
import math

import torch

from . import gb

F64 = torch.float64
C128 = torch.complex128


def _bit_reverse(N):
    bits = int(math.log2(N))
    return torch.tensor([int(format(i, "0%db" % bits)[::-1], 2) for i in range(N)], dtype=torch.int64)


def fft_radix2(s):
    """S_k = sum_n s_n exp(-2 pi i k n / N), k = 0..N-1, over the last axis (N a power of two)."""
    N = s.shape[-1]
    if N & (N - 1):
        raise ValueError("N must be a power of two")
    x = s[..., _bit_reverse(N)]
    h = 1
    while h < N:
        k = torch.arange(h, dtype=F64)
        w = torch.exp((-1j * math.pi / h) * k.to(C128))           # exp(-2 pi i k / 2h)
        x = x.reshape(*s.shape[:-1], N // (2 * h), 2, h)
        a, b = x[..., 0, :], x[..., 1, :] * w
        x = torch.stack((a + b, a - b), dim=-2).reshape(*s.shape[:-1], N)
        h *= 2
    return x


def template_fft(theta, N, T):
    """gb.template with the radix-2 FFT: q, hA, hE on bins q - N/2 .. q + N/2 - 1."""
    q, sA, sE = gb.slow_part(theta, N, T)
    scale = T / (2.0 * N)
    centre = lambda s: torch.roll(fft_radix2(s), N // 2, dims=-1)     # m = -N/2 .. N/2 - 1
    return q, scale * centre(sA), scale * centre(sE)


def loglik_fft(windows, dA, dE, wA, wE, theta, T, chunk=2048):
    """gb.loglik with template_fft: logL, dh, hh per candidate row."""
    theta = torch.as_tensor(theta, dtype=F64)
    dA, dE = torch.as_tensor(dA, dtype=C128), torch.as_tensor(dE, dtype=C128)
    wA, wE = torch.as_tensor(wA, dtype=F64), torch.as_tensor(wE, dtype=F64)
    n_total = theta.shape[0]
    logL = torch.zeros(n_total, dtype=F64)
    DH = torch.zeros(n_total, dtype=F64)
    HH = torch.zeros(n_total, dtype=F64)
    for (k0, W, N, doff, coff, nc) in windows:
        sl = slice(doff, doff + W)
        for c0 in range(coff, coff + nc, chunk):
            c1 = min(c0 + chunk, coff + nc)
            q, hA, hE = template_fft(theta[c0:c1], N, T)
            dh, hh, dd = gb.window_inner_products(k0, dA[sl], dE[sl], wA[sl], wE[sl], q, hA, hE, T)
            logL[c0:c1] = dh - 0.5 * hh - 0.5 * dd
            DH[c0:c1] = dh
            HH[c0:c1] = hh
    return logL, DH, HH
