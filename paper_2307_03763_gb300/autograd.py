"""torch.autograd interface of the likelihood: forward by gb_loglik, backward by
the adjoint kernel gb_loglik_grad, which recomputes the template instead of
saving it (only theta is kept for the backward pass)."""
import torch


class LogLikelihood(torch.autograd.Function):
    """logL(theta) per candidate; d(sum w logL)/d theta = w * gb_loglik_grad."""

    @staticmethod
    def forward(ctx_, lib_ctx, windows, dA, dE, wA, wE, theta, prec):
        logL, _, _ = lib_ctx.loglik(windows, dA, dE, wA, wE, theta.detach().contiguous(), prec=prec)
        ctx_.save_for_backward(theta)
        ctx_.lib = (lib_ctx, windows, dA, dE, wA, wE, prec)
        return logL

    @staticmethod
    def backward(ctx_, grad_out):
        (theta,) = ctx_.saved_tensors
        lib_ctx, windows, dA, dE, wA, wE, prec = ctx_.lib
        _, g = lib_ctx.loglik_grad(windows, dA, dE, wA, wE, theta.detach().contiguous(), prec=prec)
        return None, None, None, None, None, None, g * grad_out[:, None], None


def loglik(lib_ctx, windows, dA, dE, wA, wE, theta, prec="mixed"):
    """Differentiable batched log-likelihood (gradient with respect to theta only)."""
    return LogLikelihood.apply(lib_ctx, windows, dA, dE, wA, wE, theta, prec)


def observed_fisher(lib_ctx, windows, dA, dE, wA, wE, theta, prec="fp64", rel=1e-5):
    """Observed information -d^2 logL/d theta^2 at one parameter set per window,
    by central differences of the adjoint gradient (16 gradients per window in
    one batched call); returns (n_win, 8, 8), symmetrised.

    windows: (k0, W, N, data_off, _, _) per window; theta: (n_win, 8) device.
    Step per parameter: rel times its natural scale (1/T, 1/T^2, 1 rad, A).
    The entries span ~70 decades in these units: invert S F S with
    S = diag(1/T, 1/T^2, 1, 1, A, 1, 1, 1), not F itself.
    """
    n_win = theta.shape[0]
    T = lib_ctx.T_obs
    scale = torch.tensor([1 / T, 1 / T ** 2, 1, 1, 0, 1, 1, 1], dtype=torch.float64, device=theta.device)
    step = rel * scale.expand(n_win, 8).clone()
    step[:, 4] = rel * theta[:, 4].abs()
    eye = torch.eye(8, dtype=torch.float64, device=theta.device)
    pts = theta[:, None, None, :] + torch.stack([eye, -eye], 0)[None] * step[:, None, None, :]   # (w, 2, 8, 8)
    pts = pts.reshape(n_win * 16, 8).contiguous()
    wins = [(k0, W, N, doff, 16 * w, 16) for w, (k0, W, N, doff, _, _) in enumerate(windows)]
    _, g = lib_ctx.loglik_grad(wins, dA, dE, wA, wE, pts, prec=prec)
    g = g.reshape(n_win, 2, 8, 8)
    H = (g[:, 0] - g[:, 1]) / (2 * step[:, :, None])        # H[w, i, j] = d g_j / d theta_i
    F = -0.5 * (H + H.transpose(1, 2))
    return F


def expected_fisher(lib_ctx, windows, wA, wE, theta, prec="fp64", rel=1e-5):
    """Fisher matrix F_ij = <d_i h|d_j h> (Eq. 13, read with h in place of the
    garbled p(d|theta)) at one parameter set per window; returns (n_win, 8, 8).

    It is the observed information of noise-free data d = h(theta) on each
    window: -d2 logL = <d_i h|d_j h> - <d - h|d_i d_j h>, and the second term
    vanishes there.  The data are the FP64 waveforms of theta placed on the
    windows' bins; the rest is observed_fisher.
    """
    dev = theta.device
    n_bins = wA.shape[0]
    dA = torch.zeros(n_bins, dtype=torch.complex128, device=dev)
    dE = torch.zeros(n_bins, dtype=torch.complex128, device=dev)
    for N in sorted({w[2] for w in windows}):
        sel = [i for i, w in enumerate(windows) if w[2] == N]
        hA, hE, q = lib_ctx.waveform(theta[sel].contiguous(), N, "fp64")
        k0 = torch.as_tensor([windows[i][0] for i in sel], device=dev)
        W = torch.as_tensor([windows[i][1] for i in sel], device=dev)
        off = torch.as_tensor([windows[i][3] for i in sel], device=dev)
        loc = q[:, None] - N // 2 + torch.arange(N, device=dev)[None, :] - k0[:, None]
        ok = (loc >= 0) & (loc < W[:, None])
        idx = (off[:, None] + loc)[ok]
        dA[idx] = hA[ok]
        dE[idx] = hE[ok]
    return observed_fisher(lib_ctx, windows, dA, dE, wA, wE, theta, prec=prec, rel=rel)


def newton_polish(lib_ctx, windows, dA, dE, wA, wE, theta, iters=6, prec="mixed", lam0=1e-3):
    """Local maximisation of logL from one point per window (the gradient
    polish that stands in for Alg. 2's SLSQP step): Levenberg-Marquardt
    steps (F + lam diag F) d = g with the adjoint gradient g and the observed
    Fisher matrix F, solved in natural units (1/T, 1/T^2, rad, A); a step is
    taken only where it raises logL, else lam grows tenfold.  Returns the
    polished theta (n_win, 8) and its logL.  The likelihood, gradient and
    Fisher matrices come from the library; the 8x8 solves run on the host."""
    import numpy as np
    T = lib_ctx.T_obs
    th = theta.clone()
    n = th.shape[0]
    wins = [(k0, W, N, doff, w, 1) for w, (k0, W, N, doff, _, _) in enumerate(windows)]
    logL, g = lib_ctx.loglik_grad(wins, dA, dE, wA, wE, th, prec=prec)
    lam = np.full(n, lam0)
    for _ in range(int(iters)):
        F = observed_fisher(lib_ctx, windows, dA, dE, wA, wE, th, prec=prec).cpu().numpy()
        s = np.ones((n, 8))
        s[:, 0], s[:, 1], s[:, 4] = 1.0 / T, 1.0 / T ** 2, np.abs(th[:, 4].cpu().numpy())
        Fs = F * s[:, :, None] * s[:, None, :]
        gs = g.cpu().numpy() * s
        A = Fs + lam[:, None, None] * np.eye(8)[None] * np.maximum(np.abs(np.diagonal(Fs, axis1=1, axis2=2)),
                                                                     1e-12)[:, :, None]
        ok = np.all(np.isfinite(A), axis=(1, 2)) & np.all(np.isfinite(gs), axis=1)
        d = np.zeros((n, 8))
        if ok.any():
            try:
                d[ok] = np.linalg.solve(A[ok], gs[ok][:, :, None])[:, :, 0]
            except np.linalg.LinAlgError:
                # an indefinite observed Fisher matrix made some system singular:
                # solve one by one, no step where singular (lam then grows)
                for i in np.nonzero(ok)[0]:
                    try:
                        d[i] = np.linalg.solve(A[i], gs[i])
                    except np.linalg.LinAlgError:
                        d[i] = 0.0
        d = np.where(np.isfinite(d), d, 0.0)
        step = torch.as_tensor(d * s, device=th.device)
        trial = th + step
        lt, gt = lib_ctx.loglik_grad(wins, dA, dE, wA, wE, trial, prec=prec)
        better = (lt > logL) & torch.isfinite(lt)
        th = torch.where(better[:, None], trial, th)
        g = torch.where(better[:, None], gt, g)
        logL = torch.where(better, lt, logL)
        b = better.cpu().numpy()
        lam = np.where(b, np.maximum(lam / 10.0, 1e-6), lam * 10.0)
    return th, logL
