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
    refit is a Gaussian (``gb_gauss_refit``): the mean and covariance of the
    visited states (weighted by the steps spent in each), the sample
    covariance widened by ``inflate`` and blended with the current proposal's
    by the number of accepted moves against the pseudo-count ``kappa``, all
    scaled by the ratio of the next temperature to this one (the tempered
    target's variance scales with T), regularised in the first round's
    whitened metric.  Every step runs on the device, so
    the whole ladder is captured once in a CUDA graph and replayed; each
    replay starts again from the initial proposal with new draws.  A good
    initial proposal is the Fisher covariance times the first temperature
    (the tempered target's width), slightly widened.
    """

    def __init__(self, ctx, windows, dA, dE, wA, wE, mean, cov, n, seed=1, temperatures=(15, 10, 5, 3, 2, 1),
                 prec="mixed", inflate=1.44, kappa=16.0, floor=1e-4):
        self.ctx = ctx
        self.kappa = float(kappa)
        self.rounds = PosteriorRounds(ctx, windows, dA, dE, wA, wE, mean, cov, n, seed=seed, prec=prec)
        self.temperatures = [float(t) for t in temperatures]
        self.inflate = float(inflate)
        self.floor = float(floor)
        self.mean0 = self.rounds.mean.clone()
        self.chol0 = self.rounds.chol.clone()
        self.graph = None

    def _ladder(self):
        r = self.rounds
        r.mean.copy_(self.mean0)
        r.chol.copy_(self.chol0)
        for k, T in enumerate(self.temperatures):
            r.temperature.fill_(T)
            r._round()
            if k + 1 < len(self.temperatures):
                self.ctx.gauss_refit(r.theta, r.chain, self.chol0, self.temperatures[k + 1] / T, self.inflate,
                                     self.kappa, self.floor, out=(r.mean, r.chol))

    def run(self, graph=False):
        """One posterior: all temperatures from the initial proposal; the
        buffers of ``self.rounds`` hold the last (T = 1) round.  With graph,
        the first call runs the ladder eagerly and captures it; later calls
        replay the capture."""
        if not graph:
            self._ladder()
            return self
        if self.graph is None:
            self._ladder()
            self.graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(self.graph):
                self._ladder()
            return self
        self.graph.replay()
        return self
