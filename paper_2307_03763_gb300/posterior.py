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
        cov = torch.as_tensor(cov, dtype=torch.float64, device=dev).reshape(self.nw, 8, 8)
        self.chol = torch.linalg.cholesky(cov).contiguous()
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
