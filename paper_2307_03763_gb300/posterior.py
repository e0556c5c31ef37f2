"""Posterior rounds of the independence sampler on the device (Alg. 4 inner body).

One round is three library calls on the current stream: draw n Gaussian
proposals per window (``gb_draw_gaussian``), evaluate them all
(``gb_loglik``), and build one chain per window (``gb_mh_independence``).
The draws are counted on the device, so two rounds captured once in a CUDA
graph can be replayed to run many rounds.  The proposal of a round is
N(mean_w, cov_w) per window (``PosteriorRounds``, ``AnnealedPosterior``) or,
as the paper describes Alg. 4, uniform over a reduced box at the first
temperature and paired 2-D kernel-density estimates of the previous
temperature's chain afterwards (``KDEPosterior``).  The module orders calls,
owns buffers and factors the 8x8 proposal covariances once at set-up.
"""
import math

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


def reduced_box(mle, sigma, prior_lo, prior_hi):
    """The reduced parameter space of Sec. III.G for each window: theta_MLE
    +- 4 sigma, f0 +- sigma_f, fdot over its whole prior range, psi +- pi/1000,
    phi0 +- 2 pi/1000, the non-periodic ranges cut to the prior box.
    mle, sigma: (n_win, 8); prior_lo, prior_hi: (n_win, 8) or (8,).
    Returns (n_win, 16) boxes lo[8], hi[8]."""
    mle = np.atleast_2d(np.asarray(mle, dtype=np.float64))
    sigma = np.atleast_2d(np.asarray(sigma, dtype=np.float64))
    plo = np.broadcast_to(np.asarray(prior_lo, dtype=np.float64), mle.shape)
    phi = np.broadcast_to(np.asarray(prior_hi, dtype=np.float64), mle.shape)
    half = 4.0 * sigma
    half[:, 0] = sigma[:, 0]
    half[:, 6] = math.pi / 1000
    half[:, 7] = 2 * math.pi / 1000
    lo, hi = mle - half, mle + half
    lo[:, 1], hi[:, 1] = plo[:, 1], phi[:, 1]
    lo[:, :6] = np.maximum(lo[:, :6], plo[:, :6])
    hi[:, :6] = np.minimum(hi[:, :6], phi[:, :6])
    return np.concatenate([lo, hi], axis=1)


class KDEPosterior:
    """Alg. 4 as the paper describes it (Sec. III.G): a temperature ladder
    (15, 10, 5, 3, 2, 1 by default) of n proposals per window and
    temperature.  The first temperature draws uniformly from each window's
    reduced box; after each temperature the chain's states are smoothed into
    paired two-dimensional kernel-density estimates, (f0, fdot),
    (lambda, beta), (A, iota), which are the next temperature's proposal
    (``gb_kde_build`` / ``gb_kde_draw``), psi and phi0 staying uniform over
    their narrow ranges.  Each estimate is a grid x grid table over the
    chain's range on each axis (widened by three bandwidths, inside the box),
    mixed with a uniform floor so that no cell is left out.

    Every step runs on the device; with graph=True the ladder is captured
    once and replayed, each replay a new posterior from the uniform start.
    box: (n_win, 16) reduced boxes (``reduced_box``)."""

    def __init__(self, ctx, windows, dA, dE, wA, wE, box, n, seed=1, temperatures=(15, 10, 5, 3, 2, 1),
                 prec="mixed", grid=64, floor=0.01, literal=False):
        self.ctx = ctx
        dev = ctx.device
        self.nw = len(windows)
        self.n = int(n)
        self.seed = int(seed)
        self.prec = prec
        self.literal = literal
        self.grid = int(grid)
        self.floor = float(floor)
        self.temperatures = [float(t) for t in temperatures]
        self.windows = [(k0, W, N, doff, w * self.n, self.n) for w, (k0, W, N, doff, _, _) in enumerate(windows)]
        self.data = (dA, dE, wA, wE)
        self.box = torch.as_tensor(np.asarray(box, dtype=np.float64).reshape(self.nw, 16), device=dev).contiguous()
        GG = self.grid * self.grid
        flat = torch.arange(1, GG + 1, dtype=torch.float64, device=dev) / GG   # uniform over the box
        self.flat = flat.expand(self.nw, 3, GG).contiguous()
        self.cdf = self.flat.clone()
        b = self.box
        self.box_ext = torch.stack([torch.stack([b[:, dx], b[:, 8 + dx], b[:, dy], b[:, 8 + dy]], dim=1)
                                    for dx, dy in ((0, 1), (3, 2), (4, 5))], dim=1).contiguous()
        self.ext = self.box_ext.clone()
        m = self.nw * self.n
        self.theta = torch.empty((m, 8), dtype=torch.float64, device=dev)
        self.log_g = torch.empty((self.nw, self.n), dtype=torch.float64, device=dev)
        self.log_u = torch.empty((self.nw, self.n), dtype=torch.float64, device=dev)
        self.logL = torch.empty(m, dtype=torch.float64, device=dev)
        self.chain = torch.empty((self.nw, self.n), dtype=torch.int32, device=dev)
        self.accepted = torch.empty(self.nw, dtype=torch.int32, device=dev)
        self.temperature = torch.empty(self.nw, dtype=torch.float64, device=dev)
        self.rounds = torch.zeros(2, dtype=torch.int64, device=dev)
        self.graph = None

    def _ladder(self):
        c = self.ctx
        self.cdf.copy_(self.flat)
        self.ext.copy_(self.box_ext)
        K = len(self.temperatures)
        for k, T in enumerate(self.temperatures):
            s = k % 2
            self.temperature.fill_(T)
            c.kde_draw(self.box, self.grid, self.cdf, self.ext, self.n, self.seed, self.rounds[s:s + 1],
                       self.rounds[1 - s:2 - s], out=(self.theta, self.log_g, self.log_u))
            c.loglik(self.windows, *self.data, self.theta, prec=self.prec, out=(self.logL, None, None))
            c.mh_independence(self.logL.view(self.nw, self.n), self.log_g, self.log_u, self.temperature,
                              literal=self.literal, out=(self.chain, self.accepted))
            if k + 1 < K:
                c.kde_build(self.theta, self.chain, self.box, self.grid, self.floor, out=(self.cdf, self.ext))
        if K % 2:   # the next ladder reads the draw counter from slot 0
            self.rounds[0:1].copy_(self.rounds[1:2])

    def run(self, graph=False):
        """One posterior: all temperatures from the uniform start; theta,
        chain and accepted hold the last (T = 1) round.  With graph, the first
        call runs the ladder eagerly and captures it; later calls replay it."""
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
