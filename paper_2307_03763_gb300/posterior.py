"""Posterior rounds of the independence sampler on the device (Alg. 4 inner body).

One round is three library calls on the current stream: draw n Gaussian
proposals per window (``gb_draw_gaussian``), evaluate them all
(``gb_loglik``), and build one chain per window (``gb_mh_independence``).
The draws are counted on the device, so two rounds captured once in a CUDA
graph can be replayed to run many rounds.  The proposal of a round is
N(mean_w, cov_w) per window; the paper anneals and refits it with a 2-D KDE
between rounds, which is not part of this driver.  The module orders calls,
owns buffers and factors the 8x8 proposal covariances once at set-up.
"""
import numpy as np
import torch


class PosteriorRounds:
    def __init__(self, ctx, windows, dA, dE, wA, wE, mean, cov, n, seed=1, temperature=None, prec="mixed",
                 literal=False):
        self.ctx = ctx
        dev = ctx.device
        self.nw = len(windows)
        self.n = int(n)
        self.seed = int(seed)
        self.prec = prec
        self.literal = literal
        self.windows = [(k0, W, N, doff, w * self.n, self.n) for w, (k0, W, N, doff, _, _) in enumerate(windows)]
        self.data = (dA, dE, wA, wE)
        self.mean = torch.as_tensor(mean, dtype=torch.float64, device=dev).reshape(self.nw, 8).contiguous()
        # 8x8 factors on the host (no device linear-algebra library needed)
        cov = np.asarray(torch.as_tensor(cov).detach().cpu(), dtype=np.float64).reshape(self.nw, 8, 8)
        self.chol = torch.as_tensor(np.linalg.cholesky(cov), device=dev).contiguous()
        self.temperature = (torch.ones(self.nw, dtype=torch.float64, device=dev) if temperature is None else
                            torch.as_tensor(temperature, dtype=torch.float64, device=dev).contiguous())
        m = self.nw * self.n
        self.theta = torch.empty((m, 8), dtype=torch.float64, device=dev)
        self.log_g = torch.empty((self.nw, self.n), dtype=torch.float64, device=dev)
        self.log_u = torch.empty((self.nw, self.n), dtype=torch.float64, device=dev)
        self.logL = torch.empty(m, dtype=torch.float64, device=dev)
        self.chain = torch.empty((self.nw, self.n), dtype=torch.int32, device=dev)
        self.accepted = torch.empty(self.nw, dtype=torch.int32, device=dev)
        self.rounds = torch.zeros(2, dtype=torch.int64, device=dev)
        self.done = 0
        self.graph = None
        self._phase = None

    def _round(self):
        s = self.done % 2
        c = self.ctx
        c.draw_gaussian(self.mean, self.chol, self.n, self.seed, self.rounds[s:s + 1], self.rounds[1 - s:2 - s],
                        out=(self.theta, self.log_g, self.log_u))
        c.loglik(self.windows, *self.data, self.theta, prec=self.prec, out=(self.logL, None, None))
        c.mh_independence(self.logL.view(self.nw, self.n), self.log_g, self.log_u, self.temperature,
                          literal=self.literal, out=(self.chain, self.accepted))
        self.done += 1

    def run(self, rounds, graph=True):
        """Run `rounds` rounds; the buffers hold the last round's proposals, logL and chains."""
        left = int(rounds)
        while left > 0 and (self.done < 2 or not graph):
            self._round()
            left -= 1
        if left > 0:
            if self.graph is None or self._phase != self.done % 2:
                self.graph = torch.cuda.CUDAGraph()
                self._phase = self.done % 2
                done = self.done
                with torch.cuda.graph(self.graph):
                    self._round()
                    self._round()
                self.done = done
            while left >= 2:
                self.graph.replay()
                self.done += 2
                left -= 2
            if left:
                self._round()
        return self


class AnnealedPosterior:
    """Alg. 4 with a temperature ladder: one round of n proposals per
    temperature (15, 10, 5, 3, 2, 1 by default), every window's proposal
    refitted between rounds to the states its chain visited.

    The paper refits paired two-dimensional kernel density estimates; here the
    refit is a Gaussian: the mean and covariance of the visited states
    (weighted by the steps spent in each), the covariance scaled by the ratio
    of the next temperature to this one (the tempered target's variance
    scales with T), widened by ``inflate``, and floored and capped at
    ``floor`` and 1/``floor`` times the first round's in every direction.  The
    rounds run in the library (draws, likelihood, chains); the refit's
    8-dimensional means and covariances are formed with torch on the device
    and factored on the host.
    """

    def __init__(self, ctx, windows, dA, dE, wA, wE, mean, cov, n, seed=1, temperatures=(15, 10, 5, 3, 2, 1),
                 prec="mixed", inflate=1.44, floor=1e-4):
        self.rounds = PosteriorRounds(ctx, windows, dA, dE, wA, wE, mean, cov, n, seed=seed, prec=prec)
        self.temperatures = [float(t) for t in temperatures]
        self.inflate = float(inflate)
        self.floor = float(floor)
        self.L0 = self.rounds.chol.cpu().numpy()

    def _refit(self, ratio):
        r = self.rounds
        th = r.theta.view(r.nw, r.n, 8)
        idx = r.chain.long()                                              # state after every step
        states = torch.gather(th, 1, idx[:, :, None].expand(-1, -1, 8))   # (nw, n, 8): steps weigh the states
        mu = states.mean(1)
        dev = states - mu[:, None, :]
        cov = (dev.transpose(1, 2) @ dev / max(1, r.n - 1)).cpu().numpy()
        mu = np.nan_to_num(mu.cpu().numpy())
        # the next target is narrower by T_next/T in variance
        cov = ratio * self.inflate * 0.5 * (cov + cov.transpose(0, 2, 1))
        # floor and cap the eigenvalues in the first round's metric, then take
        # the lower-triangular factor with a positive diagonal from the QR
        # factors of a square root (no squaring of the condition number; the
        # natural units span ~20 decades)
        Li = np.linalg.inv(self.L0)
        M = Li @ cov @ Li.transpose(0, 2, 1)
        ev, V = np.linalg.eigh(0.5 * (M + M.transpose(0, 2, 1)))
        ev = np.clip(np.nan_to_num(ev, nan=1.0), self.floor, 1.0 / self.floor)
        S = self.L0 @ (V * np.sqrt(ev)[:, None, :])
        _, Rq = np.linalg.qr(S.transpose(0, 2, 1))
        L = Rq.transpose(0, 2, 1)
        L = L * np.sign(np.diagonal(L, axis1=1, axis2=2))[:, None, :]
        r.mean.copy_(torch.as_tensor(mu))
        r.chol.copy_(torch.as_tensor(L))

    def run(self):
        """All temperatures; the buffers of ``self.rounds`` hold the last (T = 1) round."""
        r = self.rounds
        for k, T in enumerate(self.temperatures):
            r.temperature.fill_(T)
            r.run(1, graph=False)
            if k + 1 < len(self.temperatures):
                self._refit(self.temperatures[k + 1] / T)
        return self
