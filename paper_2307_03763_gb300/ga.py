"""Genetic search of every window on the device: a thin driver over libgb.

One generation is three library calls on the current stream: the batched
likelihood of the whole population (``gb_loglik``, or ``gb_loglik_phase``
when the fitness is maximised over phi0 in closed form), the gradient at each
window's best individual (``gb_loglik_grad``, the polish step) and
``gb_ga_step`` (selection, crossover, mutation, the best individual with its
analytic amplitude, and steps along the gradient).  Two generations
(population buffers A -> B -> A) are captured once in a CUDA graph and
replayed; the random draws are counted on the device, so each replay advances
the search.  Nothing here computes: the module only allocates buffers, orders
the calls and captures them.
"""
import numpy as np
import torch

from . import api


class GASearch:
    """Maximise the SNR of every window's population (Eq. 6; A from Eq. 7).

    windows: (k0, W, N, data_off, _, _) per window; data tensors as for
    ``Context.loglik``; boxes: (n_win, 16) prior boxes (lo[8], hi[8]);
    pop: individuals per window.  The initial population is drawn uniformly
    in each box from ``seed`` (an input of the search); init (optional, one
    (k, 8) array per window, k <= pop) replaces the first k draws of a window
    by given starting points (kept inside its box).  phase=True ranks
    individuals by their SNR maximised over phi0 (the template carries phi0
    as a common factor exp(i phi0)) and rotates the best one to that phase.
    """

    def __init__(self, ctx, windows, dA, dE, wA, wE, boxes, pop, seed=1, prec="mixed", params=None, polish=True,
                 phase=True, init=None):
        self.ctx = ctx
        self.nw = len(windows)
        self.pop = int(pop)
        self.prec = prec
        self.polish = polish
        self.phase = phase
        self.seed = int(seed)
        self.windows = [(k0, W, N, doff, w * self.pop, self.pop) for w, (k0, W, N, doff, _, _) in enumerate(windows)]
        self.best_windows = [(k0, W, N, doff, w, 1) for w, (k0, W, N, doff, _, _) in enumerate(windows)]
        self.data = (dA, dE, wA, wE)
        dev = ctx.device
        boxes = np.asarray(boxes, dtype=np.float64).reshape(self.nw, 16)
        self.box = torch.as_tensor(boxes, device=dev).contiguous()
        lo, hi = boxes[:, :8], boxes[:, 8:]
        rng = np.random.default_rng(self.seed)
        th0 = lo[:, None, :] + (hi - lo)[:, None, :] * rng.uniform(size=(self.nw, self.pop, 8))
        if init is not None:
            for w, s in enumerate(init):
                s = np.asarray(s, dtype=np.float64).reshape(-1, 8)[:self.pop]
                if s.shape[0]:
                    th0[w, :s.shape[0]] = np.clip(s, lo[w], hi[w])
        n = self.nw * self.pop
        self.th = [torch.as_tensor(th0.reshape(n, 8), device=dev).contiguous(),
                   torch.empty((n, 8), dtype=torch.float64, device=dev)]
        self.logL = torch.zeros(n, dtype=torch.float64, device=dev)
        self.dh = torch.zeros(n, dtype=torch.float64, device=dev)
        self.hh = torch.zeros(n, dtype=torch.float64, device=dev)
        self.dh_im = torch.zeros(n, dtype=torch.float64, device=dev) if phase else None
        self.best = torch.zeros((self.nw, 8), dtype=torch.float64, device=dev)
        self.grad = torch.zeros((self.nw, 8), dtype=torch.float64, device=dev)
        self.gen = torch.zeros(2, dtype=torch.int64, device=dev)
        self.params = params or api.GAParams(3, 0, 0.9, 0.15, 0.02)
        self.cur = 0          # population buffer of the next generation's parents
        self.done = 0         # generations run
        self.graph = None

    def _generation(self, polish):
        src, dst = self.cur, 1 - self.cur
        slot = self.done % 2
        ctx = self.ctx
        if self.phase:
            ctx.loglik_phase(self.windows, *self.data, self.th[src], prec=self.prec,
                             out=(self.logL, self.dh, self.dh_im, self.hh))
        else:
            ctx.loglik(self.windows, *self.data, self.th[src], prec=self.prec, out=(self.logL, self.dh, self.hh))
        grad = None
        if polish:
            ctx.loglik_grad(self.best_windows, *self.data, self.best, prec=self.prec, out=(None, self.grad))
            grad = self.grad
        ctx.ga_step(self.nw, self.pop, self.th[src], self.dh, self.hh, self.box, self.seed,
                    self.gen[slot:slot + 1], self.gen[1 - slot:2 - slot], self.params, grad,
                    out=self.th[dst], best=self.best, dh_im=self.dh_im)
        self.cur = dst
        self.done += 1

    def run(self, generations, graph=True):
        """Run `generations` generations; returns the best individuals (n_win, 8) on the host."""
        left = int(generations)
        while left > 0 and (self.done < 2 or not graph):
            self._generation(self.polish and self.done > 0)
            left -= 1
        if left > 0:
            if self.graph is None or self.done % 2 != self._graph_phase:
                # capture two generations; the population and the counter slot
                # return to the state they started from
                self.graph = torch.cuda.CUDAGraph()
                self._graph_phase = self.done % 2
                cur, done = self.cur, self.done
                with torch.cuda.graph(self.graph):
                    self._generation(self.polish)
                    self._generation(self.polish)
                self.cur, self.done = cur, done
            while left >= 2:
                self.graph.replay()
                self.done += 2
                left -= 2
            if left:
                self._generation(self.polish)
        torch.cuda.current_stream(self.ctx.device).synchronize()
        return self.best.cpu().numpy()

    def best_snr(self):
        """SNR (Eq. 6) of each window's best individual."""
        _, dh, hh = self.ctx.loglik(self.best_windows, *self.data, self.best, prec=self.prec)
        return (dh / torch.sqrt(hh)).cpu().numpy()
