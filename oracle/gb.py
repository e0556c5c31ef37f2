"""Galactic-binary template, window inner products and log-likelihood, plain FP64.

TEST INFRASTRUCTURE (see the package docstring): only tests/, the smoke check
and the CPU-baseline leg of bench.py may call this.

What the paper fixes
--------------------
* log-likelihood  log p(d|theta) = -1/2 <d - s(theta) | d - s(theta)>   (Eq. 2)
* inner product   <x|y> = 4 Re int x~ y~* / S df, one-sided S           (Eq. 3)
  restricted to the analysed frequency window                           (Sec. III.D)
* sum over TDI channels, A = (Z - X)/sqrt2, E = (X - 2Y + Z)/sqrt6      (Eqs. 4-5)
* eight parameters {A, lambda, beta, f, fdot, iota, phi0, psi}, first-order
  fdot only                                                             (Sec. III, first paragraph)
* SNR rho = <d|s>/sqrt<s|s> and A_max = <d|s'>/<s'|s'>                  (Eqs. 6-7)
* multi-signal SNR rho = <d|sum s>/sqrt<sum s|sum s>                    (Eq. 11)
* scaled error delta and overlap O of a recovery against an injection   (Eqs. 19-20)

What the paper only cites (the signal model and the LISA response) is written
out here from the physics, with these readings:

R1  Parameter order theta = (f0, fdot, beta, lambda, A, iota, psi, phi0).
R2  Constants: c exact, AU = 1.495978707e11 m, year = 31 557 600 s (Julian),
    L = 2.5e9 m, f* = c / (2 pi L).
R3  Orbit: rigid equal-arm triangle on the first-order (in e = L/(2 sqrt3 AU))
    heliocentric orbit, alpha = 2 pi t / yr, spacecraft i at beta_i = 2 pi i/3:
      x_i = AU cos a + AU e/2 (cos(2a - b_i) - 3 cos b_i)
      y_i = AU sin a + AU e/2 (sin(2a - b_i) - 3 sin b_i)
      z_i = -sqrt3 AU e cos(a - b_i)
    The arm lengths of this orbit are exactly L; every delay uses L/c.
R4  Source: propagation direction k = -(cos b cos l, cos b sin l, sin b);
    u = (sin b cos l, sin b sin l, -cos b), v = (sin l, -cos l, 0);
    e+ = uu - vv, ex = uv + vu rotated by psi:
      E+ = cos2psi e+ - sin2psi ex,  Ex = sin2psi e+ + cos2psi ex;
    h_ab(t, x) = Re[ H_ab exp(i Phi(t - k.x/c)) ],  H = A+ E+ - i Ax Ex,
    A+ = A (1 + cos^2 iota), Ax = -2 A cos iota,
    Phi(xi) = 2 pi f0 xi + pi fdot xi^2 + phi0.
R5  One link, emitter i -> receiver j, unit vector n = (x_j - x_i)/|x_j - x_i|:
      y_ij = 1/2 n.[h(emission) - h(reception)].n / (1 - k.n)
    whose slowly varying complex amplitude, with f = f0 + fdot t, is
      z_ij = -i (f/2f*) sinc(X_ij) exp(-i X_ij) (n.H.n) exp(i Psi_j),
      X_ij = (f/2f*)(1 - k.n),
    Psi_j = Phi(t - k.x_j/c) - 2 pi q t / T  (the receiver's phase, heterodyned).
R6  First-generation equal-arm TDI with delay factor D = exp(-i f/f*):
      X = (1 - D^2)[(z_21 + D z_12) - (z_31 + D z_13)], Y, Z cyclically.
R7  Carrier bin q = floor(f0 T + fdot T^2/2 + 1/2) (the mid-observation
    frequency), evaluated with one IEEE rounding per operation in the order
    ((f0*T) + ((0.5*fdot)*T)*T) + 0.5; offset delta = f0*T - q.
R8  Slow part sampled at t_n = n T/N, n = 0..N-1; N-point DFT
      S_m = sum_n s_n exp(-2 pi i m n / N),  m = -N/2 .. N/2-1,
    template h~(f_{q+m}) = (T / 2N) S_m (the 1/2 because h = Re z).
R9  Discrete inner product over window bins k in [k0, k0+W):
      <x|y> = (4/T) Re sum_k w_k x_k y_k*,  w_k = 1/S_k.
    Template bins outside the window are dropped; window bins without
    template contribute only to <d|d>.
R10 logL = <d|h> - <h|h>/2 - <d|d>/2 (Eq. 2 expanded; all three restricted
    to the window).
R11 T = (X + Y + Z)/sqrt3 (Eq. 5).  The paper drops T below f*/2 = c/(4 pi L)
    because its response is suppressed there (Sec. II); a window uses T when
    its lowest frequency k0/T is at least f*/2, and its <.|.> then sums A, E
    and T.
"""
import math

import numpy as np

import torch

F64 = torch.float64
C128 = torch.complex128

C_LIGHT = 299792458.0
AU = 1.495978707e11
YEAR = 31557600.0
ARM_L = 2.5e9

PARAM_NAMES = ("f0", "fdot", "beta", "lam", "A", "iota", "psi", "phi0")

# ordered links (emitter, receiver), spacecraft numbered 0, 1, 2
LINKS = ((0, 1), (1, 0), (0, 2), (2, 0), (1, 2), (2, 1))


def transfer_frequency(L=ARM_L):
    """f* = c / (2 pi L), the transfer frequency of Sec. II (reading R2)."""
    return C_LIGHT / (2.0 * math.pi * L)


def spacecraft_positions(t, L=ARM_L, static=False):
    """Spacecraft positions x_i(t) in metres, shape (len(t), 3, 3) = [time, craft, xyz].

    Reading R3 (the paper cites the orbit model, Sec. III first paragraph).
    ``static=True`` freezes the constellation at its t = 0 position, which turns
    the response into a textbook tone (used only by tests).
    """
    t = torch.as_tensor(t, dtype=F64)
    if static:
        t = torch.zeros_like(t)
    ecc = L / (2.0 * math.sqrt(3.0) * AU)
    a = 2.0 * math.pi * t / YEAR
    craft = []
    for i in range(3):
        b = 2.0 * math.pi * i / 3.0
        x = AU * torch.cos(a) + 0.5 * AU * ecc * (torch.cos(2.0 * a - b) - 3.0 * math.cos(b))
        y = AU * torch.sin(a) + 0.5 * AU * ecc * (torch.sin(2.0 * a - b) - 3.0 * math.sin(b))
        z = -math.sqrt(3.0) * AU * ecc * torch.cos(a - b)
        craft.append(torch.stack([x, y, z], dim=-1))
    return torch.stack(craft, dim=-2)


def propagation_direction(beta, lam):
    """Unit propagation vector k of a wave from ecliptic (beta, lambda), shape (B, 3) (R4)."""
    cb = torch.cos(beta)
    return -torch.stack([cb * torch.cos(lam), cb * torch.sin(lam), torch.sin(beta)], dim=-1)


def polarisation_tensor(A, iota, psi, beta, lam):
    """Complex strain amplitude H = A+ E+ - i Ax Ex, shape (B, 3, 3) (R4)."""
    zero = torch.zeros_like(beta)
    u = torch.stack([torch.sin(beta) * torch.cos(lam), torch.sin(beta) * torch.sin(lam), -torch.cos(beta)], -1)
    v = torch.stack([torch.sin(lam), -torch.cos(lam), zero], -1)
    ep = u[:, :, None] * u[:, None, :] - v[:, :, None] * v[:, None, :]
    ex = u[:, :, None] * v[:, None, :] + v[:, :, None] * u[:, None, :]
    c2, s2 = torch.cos(2.0 * psi)[:, None, None], torch.sin(2.0 * psi)[:, None, None]
    Ep = c2 * ep - s2 * ex
    Ex = s2 * ep + c2 * ex
    Ap = (A * (1.0 + torch.cos(iota) ** 2))[:, None, None]
    Ax = (-2.0 * A * torch.cos(iota))[:, None, None]
    return Ap * Ep.to(C128) - 1j * Ax * Ex.to(C128)


def carrier_bin(f0, fdot, T):
    """Carrier bin q (int64) and offset delta = f0 T - q (R7).

    q sits at the mid-observation frequency f0 + fdot T/2; it is held fixed
    under differentiation (its derivative is zero almost everywhere).
    """
    f0T = f0 * T
    x = f0T + ((0.5 * fdot) * T) * T
    q = torch.floor(x + 0.5).detach()
    return q.to(torch.int64), f0T - q


def slow_part(theta, N, T, L=ARM_L, static=False):
    """Heterodyned TDI A and E at t_n = n T/N (R5, R6, R8; Eqs. 4-5).

    theta: (B, 8) float64 in the order of R1.  Returns q (B,), sA (B, N), sE (B, N).
    """
    q, sA, sE, _ = slow_part_aet(theta, N, T, L, static)
    return q, sA, sE


def slow_part_aet(theta, N, T, L=ARM_L, static=False):
    """Heterodyned TDI A, E and T at t_n = n T/N (R5, R6, R8, R11; Eqs. 4-5).

    Returns q (B,), sA, sE, sT (B, N)."""
    theta = torch.as_tensor(theta, dtype=F64)
    f0, fdot, beta, lam, A, iota, psi, phi0 = theta.unbind(-1)
    q, delta = carrier_bin(f0, fdot, T)
    t = torch.arange(N, dtype=F64) * (T / N)
    x = spacecraft_positions(t, L, static)                   # (N, 3, 3)
    k = propagation_direction(beta, lam)                     # (B, 3)
    H = polarisation_tensor(A, iota, psi, beta, lam)         # (B, 3, 3)
    kappa = torch.einsum("bc,nsc->bns", k, x) / C_LIGHT      # k.x_j / c, (B, N, 3)

    tt = t[None, :]
    f0c, fdc, phc = f0[:, None, None], fdot[:, None, None], phi0[:, None, None]
    t3 = tt[:, :, None]
    # Psi_j = Phi(t - k.x_j/c) - 2 pi q t/T, expanded exactly (R5)
    phase = 2.0 * math.pi * (delta[:, None, None] * t3 / T + 0.5 * fdc * t3 ** 2 - f0c * kappa
                             - fdc * t3 * kappa + 0.5 * fdc * kappa ** 2) + phc
    rx = torch.exp(1j * phase)                               # (B, N, 3)

    freq = f0[:, None] + fdot[:, None] * tt                  # (B, N)
    fstar = transfer_frequency(L)
    a = freq / (2.0 * fstar)
    z = {}
    for (i, j) in LINKS:
        n = x[:, j, :] - x[:, i, :]
        n = n / torch.linalg.vector_norm(n, dim=-1, keepdim=True)          # (N, 3)
        kn = torch.einsum("bc,nc->bn", k, n)
        nc = n.to(C128)
        G = torch.einsum("nr,brs,ns->bn", nc, H, nc)
        X = a * (1.0 - kn)
        z[(i, j)] = -1j * a * torch.sinc(X / math.pi) * torch.exp(-1j * X) * G * rx[:, :, j]

    D = torch.exp(-1j * freq / fstar)
    one_m_D2 = 1.0 - D * D

    def michelson(c, p, r):
        # round trips c->p->c and c->r->c, both read at corner c (R6)
        return one_m_D2 * ((z[(p, c)] + D * z[(c, p)]) - (z[(r, c)] + D * z[(c, r)]))

    Xc = michelson(0, 1, 2)
    Yc = michelson(1, 2, 0)
    Zc = michelson(2, 0, 1)
    sA = (Zc - Xc) / math.sqrt(2.0)
    sE = (Xc - 2.0 * Yc + Zc) / math.sqrt(6.0)
    sT = (Xc + Yc + Zc) / math.sqrt(3.0)
    return q, sA, sE, sT


def dft_centered(s):
    """Naive DFT S_m = sum_n s_n exp(-2 pi i m n/N) for m = -N/2..N/2-1 (R8).

    The product m*n is reduced modulo N in exact integer arithmetic before the
    exponential so that every twiddle is correctly rounded.
    """
    N = s.shape[-1]
    m = torch.arange(-(N // 2), N // 2, dtype=torch.int64)
    n = torch.arange(N, dtype=torch.int64)
    r = torch.remainder(m[:, None] * n[None, :], N).to(F64)
    M = torch.exp((-2.0j * math.pi / N) * r.to(C128))
    return s @ M.transpose(0, 1)


def template(theta, N, T, L=ARM_L, static=False):
    """Frequency-domain A/E template on bins q - N/2 .. q + N/2 - 1 (R8).

    Returns q (B,), hA (B, N), hE (B, N), entry m' standing for bin q - N/2 + m'.
    This is what the waveform entry point of the library returns.
    """
    q, sA, sE = slow_part(theta, N, T, L, static)
    scale = T / (2.0 * N)
    return q, scale * dft_centered(sA), scale * dft_centered(sE)


def template_aet(theta, N, T, L=ARM_L, static=False):
    """template() with the T channel: q, hA, hE, hT (R8, R11)."""
    q, sA, sE, sT = slow_part_aet(theta, N, T, L, static)
    scale = T / (2.0 * N)
    return q, scale * dft_centered(sA), scale * dft_centered(sE), scale * dft_centered(sT)


def uses_t(k0, T, L=ARM_L):
    """R11: the window's lowest frequency k0/T is at least f*/2."""
    return k0 / T >= 0.5 * transfer_frequency(L)


def window_inner_products(k0, dA, dE, wA, wE, q, hA, hE, T):
    """<d|h>, <h|h> over the window bins, and <d|d> (R9; Eqs. 3-4, Sec. III.D).

    dA, dE: (W,) complex data on bins k0..k0+W-1; wA, wE: (W,) = 1/S;
    q: (B,) carrier bins; hA, hE: (B, N) templates.  Returns dh (B,), hh (B,), dd ().
    """
    W = dA.shape[0]
    N = hA.shape[-1]
    j = q[:, None] - N // 2 + torch.arange(N, dtype=torch.int64)[None, :] - k0
    inside = (j >= 0) & (j < W)
    jc = j.clamp(0, max(W - 1, 0))
    dh = torch.zeros(q.shape[0], dtype=F64)
    hh = torch.zeros(q.shape[0], dtype=F64)
    dd = torch.zeros((), dtype=F64)
    if W > 0:
        for d, w, h in ((dA, wA, hA), (dE, wE, hE)):
            dk, wk = d[jc], w[jc]
            dh = dh + torch.where(inside, wk * (dk * h.conj()).real, 0.0).sum(-1)
            hh = hh + torch.where(inside, wk * (h.real ** 2 + h.imag ** 2), 0.0).sum(-1)
            dd = dd + (w * (d.real ** 2 + d.imag ** 2)).sum()
    return (4.0 / T) * dh, (4.0 / T) * hh, (4.0 / T) * dd


def loglik(windows, dA, dE, wA, wE, theta, T, L=ARM_L, chunk=2048):
    """Batched log-likelihood over windows (Eq. 2 with R9, R10).

    windows: sequence of (k0, W, N, data_off, cand_off, n_cand); the data of
    window w are entries data_off .. data_off+W-1 of dA, dE, wA, wE and its
    candidates are rows cand_off .. cand_off+n_cand-1 of theta (n_total, 8).
    Returns logL, dh, hh, each (n_total,) float64.  Rows that belong to no
    window are left at zero.
    """
    theta = torch.as_tensor(theta, dtype=F64)
    dA, dE = torch.as_tensor(dA, dtype=C128), torch.as_tensor(dE, dtype=C128)
    wA, wE = torch.as_tensor(wA, dtype=F64), torch.as_tensor(wE, dtype=F64)
    n_total = theta.shape[0]
    parts = {}
    for (k0, W, N, doff, coff, nc) in windows:
        sl = slice(doff, doff + W)
        for c0 in range(coff, coff + nc, chunk):
            c1 = min(c0 + chunk, coff + nc)
            q, hA, hE = template(theta[c0:c1], N, T, L)
            dh, hh, dd = window_inner_products(k0, dA[sl], dE[sl], wA[sl], wE[sl], q, hA, hE, T)
            parts[c0] = (c0, c1, dh - 0.5 * hh - 0.5 * dd, dh, hh)
    logL = torch.zeros(n_total, dtype=F64)
    DH = torch.zeros(n_total, dtype=F64)
    HH = torch.zeros(n_total, dtype=F64)
    if parts:
        idx = torch.cat([torch.arange(p[0], p[1]) for p in parts.values()])
        logL = logL.index_put((idx,), torch.cat([p[2] for p in parts.values()]))
        DH = DH.index_put((idx,), torch.cat([p[3] for p in parts.values()]))
        HH = HH.index_put((idx,), torch.cat([p[4] for p in parts.values()]))
    return logL, DH, HH


def loglik_aet(windows, dA, dE, dT, wA, wE, wT, theta, T, L=ARM_L, chunk=2048):
    """loglik() with the T channel in the windows above f*/2 (R11); dT, wT
    alongside dA, wA.  Returns logL, dh, hh."""
    theta = torch.as_tensor(theta, dtype=F64)
    dA, dE, dT = (torch.as_tensor(x, dtype=C128) for x in (dA, dE, dT))
    wA, wE, wT = (torch.as_tensor(x, dtype=F64) for x in (wA, wE, wT))
    n_total = theta.shape[0]
    logL = torch.zeros(n_total, dtype=F64)
    DH = torch.zeros(n_total, dtype=F64)
    HH = torch.zeros(n_total, dtype=F64)
    for (k0, W, N, doff, coff, nc) in windows:
        sl = slice(doff, doff + W)
        for c0 in range(coff, coff + nc, chunk):
            c1 = min(c0 + chunk, coff + nc)
            q, hA, hE, hT = template_aet(theta[c0:c1], N, T, L)
            dh, hh, dd = window_inner_products(k0, dA[sl], dE[sl], wA[sl], wE[sl], q, hA, hE, T)
            if uses_t(k0, T, L):
                dht, hht, ddt = window_inner_products(k0, dT[sl], dT[sl] * 0, wT[sl], wT[sl] * 0, q, hT,
                                                      hT * 0, T)
                dh, hh, dd = dh + dht, hh + hht, dd + ddt
            logL[c0:c1] = dh - 0.5 * hh - 0.5 * dd
            DH[c0:c1] = dh
            HH[c0:c1] = hh
    return logL, DH, HH


def loglik_grad_aet(windows, dA, dE, dT, wA, wE, wT, theta, T, L=ARM_L, chunk=2048):
    """loglik_grad() of loglik_aet(): the T channel in windows above f*/2 (R11)."""
    th = torch.as_tensor(theta, dtype=F64).detach().clone().requires_grad_(True)
    logL, _, _ = loglik_aet(windows, dA, dE, dT, wA, wE, wT, th, T, L, chunk)
    logL.sum().backward()
    return logL.detach(), th.grad.detach()


def loglik_grad(windows, dA, dE, wA, wE, theta, T, L=ARM_L, chunk=2048):
    """d logL / d theta for every candidate row, by reverse-mode autodiff of ``loglik``.

    Each logL depends on its own row only, so the gradient of the sum is the
    per-row gradient.  q is held fixed (R7).  Returns logL (n,), grad (n, 8).
    """
    th = torch.as_tensor(theta, dtype=F64).detach().clone().requires_grad_(True)
    logL, _, _ = loglik(windows, dA, dE, wA, wE, th, T, L, chunk)
    logL.sum().backward()
    return logL.detach(), th.grad.detach()


def snr(dh, hh):
    """rho = <d|s> / sqrt(<s|s>), independent of A (Eq. 6)."""
    return dh / torch.sqrt(hh)


def amplitude_max(A, dh, hh):
    """A_max = <d|s'>/<s'|s'> with s' the unit-amplitude template (Eq. 7).

    With h = A s', <d|s'> = dh/A and <s'|s'> = hh/A^2, so A_max = A dh/hh.
    """
    return A * dh / hh


def _on_window(theta, k0, W, N, T, L=ARM_L):
    """Templates of theta (K, 8) restricted to window bins k0..k0+W-1 (zero
    where a template has no bin): (K, W) complex A and E (R8, R9)."""
    q, hA, hE = template(theta, N, T, L)
    K = theta.shape[0]
    outA = torch.zeros((K, W), dtype=C128)
    outE = torch.zeros((K, W), dtype=C128)
    j = q[:, None] - N // 2 + torch.arange(N, dtype=torch.int64)[None, :] - k0
    inside = (j >= 0) & (j < W)
    for k in range(K):
        outA[k, j[k][inside[k]]] = hA[k][inside[k]]
        outE[k, j[k][inside[k]]] = hE[k][inside[k]]
    return outA, outE


def _inner(xA, xE, yA, yE, wA, wE, T):
    """<x|y> over window bins (R9): (4/T) Re sum_k w_k x_k y_k*, both channels."""
    return (4.0 / T) * ((wA * (xA * yA.conj()).real).sum(-1) + (wE * (xE * yE.conj()).real).sum(-1))


def snr_multi(windows, dA, dE, wA, wE, theta, T, L=ARM_L):
    """Multi-signal SNR (Eq. 11, Sec. III.D) of each window's sources, and its parts.

    Window w = (k0, W, N, data_off, cand_off, n_cand) holds the K = n_cand
    sources theta[cand_off:cand_off+K].  Eq. 11 as printed: the sum of the
    sources' templates S, then rho = <d|S> / sqrt(<S|S>).  Also returned, for
    the same window: the Gram matrix G_ij = <s_i|s_j> and b_i = <d|s_i>.
    Returns (rho (n_win,), [G_w (K, K)], b (n_rows,)).
    """
    theta = torch.as_tensor(theta, dtype=F64)
    dA, dE = torch.as_tensor(dA, dtype=C128), torch.as_tensor(dE, dtype=C128)
    wA, wE = torch.as_tensor(wA, dtype=F64), torch.as_tensor(wE, dtype=F64)
    rho = torch.full((len(windows),), float("nan"), dtype=F64)
    grams = []
    b = torch.zeros(theta.shape[0], dtype=F64)
    for w, (k0, W, N, doff, coff, nc) in enumerate(windows):
        sl = slice(doff, doff + W)
        if nc == 0:
            grams.append(torch.zeros((0, 0), dtype=F64))
            continue
        sA, sE = _on_window(theta[coff:coff + nc], k0, W, N, T, L)
        SA, SE = sA.sum(0), sE.sum(0)                      # the sum of the templates
        num = _inner(dA[sl], dE[sl], SA, SE, wA[sl], wE[sl], T)
        den = _inner(SA, SE, SA, SE, wA[sl], wE[sl], T)
        rho[w] = num / torch.sqrt(den)
        G = torch.empty((nc, nc), dtype=F64)
        for i in range(nc):
            for j in range(nc):
                G[i, j] = _inner(sA[i], sE[i], sA[j], sE[j], wA[sl], wE[sl], T)
        grams.append(G)
        b[coff:coff + nc] = torch.stack([_inner(dA[sl], dE[sl], sA[i], sE[i], wA[sl], wE[sl], T)
                                         for i in range(nc)])
    return rho, grams, b


def match_metrics(window, wA, wE, theta_rec, theta_inj, T, L=ARM_L):
    """Scaled error (Eq. 19) and overlap (Eq. 20) of a recovered source
    against an injected one (Sec. IV), both templates of length N on the
    window (k0, W, N, data_off, ...):
        delta = <s_rec - s_inj|s_rec - s_inj> / <s_rec|s_rec>,
        O = <s_rec|s_inj> / sqrt(<s_rec|s_rec> <s_inj|s_inj>)."""
    k0, W, N, doff = window[:4]
    wA = torch.as_tensor(wA, dtype=F64)[doff:doff + W]
    wE = torch.as_tensor(wE, dtype=F64)[doff:doff + W]
    th = torch.as_tensor(np.stack([np.asarray(theta_rec), np.asarray(theta_inj)]), dtype=F64)
    sA, sE = _on_window(th, k0, W, N, T, L)
    dA, dE = sA[0] - sA[1], sE[0] - sE[1]
    rr = _inner(sA[0], sE[0], sA[0], sE[0], wA, wE, T)
    ii = _inner(sA[1], sE[1], sA[1], sE[1], wA, wE, T)
    ri = _inner(sA[0], sE[0], sA[1], sE[1], wA, wE, T)
    delta = _inner(dA, dE, dA, dE, wA, wE, T) / rr
    return delta, ri / torch.sqrt(rr * ii)
