"""Full-band search over libgb: synthetic galaxy, genetic search in every
window, and an independence-sampler posterior for every recovered source.

The paper's global fit cuts the band into segments (Alg. 1), searches each
segment for the loudest binaries with subtract-and-repeat (Alg. 2-3, there
with differential evolution and SLSQP), and draws a 10,000-proposal
posterior per recovered source (Alg. 4).  This driver runs that flow with the
library's kernels, batched over all windows at once:

  synthesis  templates of every injected source from ``gb_waveform`` (FP64),
             scattered into the contiguous band on top of the noise, then
             copied into the windows;
  search     per round, one ``GASearch`` over all windows, f0 over each
             padded segment (gradient-polished elites, generations replayed
             from a CUDA graph), then Levenberg-Marquardt steps from each
             window's best individual (adjoint gradient, observed Fisher
             matrix); the result counts as found when its SNR (Eq. 6) on the
             window's residual passes the threshold, and as recovered when its
             f0 also lies in the unpadded segment (Alg. 2's theta_in; a
             signal in the padding belongs to the neighbour and is only
             subtracted);
  posterior  for the round's recovered sources, Alg. 4: the six-temperature
             ladder (10,000 proposals per temperature) of
             ``AnnealedPosterior`` (default: Gaussian proposals from the
             observed Fisher matrix of the adjoint gradient, refitted between
             temperatures) or of ``KDEPosterior`` (posterior="kde": uniform
             over the reduced box, then paired 2-D KDEs, as the paper
             describes it; from search optima its final-round acceptance is
             far lower);
  subtract   the recovered templates (``gb_waveform``) leave the window data
             before the next round.

Windows keep their own copies of the data; within a run a recovered source is
removed from its window only.  scheme="evenodd" runs the paper's three runs
over even and odd segments (Table 2): between runs the other parity's
signals are subtracted from the whole band and the window copies refreshed.
noise="median" replaces each searched window's weights by its median
periodogram (Sec. III.C) before every round.  The module orders calls,
moves data and keeps statistics; the arithmetic runs in the library.
"""
import math
import time

import numpy as np
import torch

from . import api
from . import autograd as gbag
from . import workloads as wk
from .ga import GASearch
from .posterior import AnnealedPosterior, KDEPosterior, reduced_box

# fixed parts of every window's search box (the f0 range is the segment's)
_LO = np.array([0.0, 0.0, -np.pi / 2, -np.pi, 1e-24, 0.0, 0.0, 0.0])
_HI = np.array([0.0, 0.0, np.pi / 2, np.pi, 1e-20, np.pi, np.pi, 2 * np.pi])


def _sync(dev):
    torch.cuda.synchronize(dev)
    return time.perf_counter()


class FullBand:
    """sources: (n, 8) injected parameters; layout: ``workloads.fullband_layout``."""

    def __init__(self, ctx, sources, layout, T, seed=1, prec="mixed"):
        if ctx.T_obs != float(T):
            raise ValueError("the context's observation time (%g s) differs from T (%g s): its orbit tables and "
                             "templates belong to T_obs" % (ctx.T_obs, T))
        self.ctx = ctx
        self.dev = ctx.device
        self.src = np.asarray(sources, dtype=np.float64)
        self.layout = list(layout)
        self.T = float(T)
        self.seed = int(seed)
        self.prec = prec
        self.n_win = len(self.layout)
        self.k_lo = min(k0 for k0, N, a, b in self.layout)
        self.k_hi = max(k0 + N for k0, N, a, b in self.layout)
        offs = np.cumsum([0] + [N for _, N, _, _ in self.layout])
        self.doff = offs[:-1]
        self.n_bins = int(offs[-1])
        self.stats = {}

    # -- synthesis ---------------------------------------------------------

    def _scatter(self, target, k_base, theta, N, sign):
        """target (bins,) complex128 += sign * templates of theta (B, 8) at N,
        placed at absolute bins q - N/2 + m minus k_base (outside: dropped)."""
        for i in range(0, theta.shape[0], 16384):
            th = theta[i:i + 16384]
            hA, hE, q = self.ctx.waveform(th, N, "fp64")
            idx = (q[:, None] - N // 2 + torch.arange(N, device=self.dev)[None, :] - k_base).reshape(-1)
            ok = (idx >= 0) & (idx < target[0].shape[0])
            for tgt, h in zip(target, (hA, hE)):
                v = torch.view_as_real(h.reshape(-1))[ok] * sign
                torch.view_as_real(tgt).index_add_(0, idx[ok], v)

    def synthesize(self, noise_seed=None):
        t0 = _sync(self.dev)
        rng = np.random.default_rng(self.seed if noise_seed is None else noise_seed)
        nA, nE, w = wk.band_noise(self.k_lo, self.k_hi, self.T, rng)
        bandA = torch.as_tensor(nA, device=self.dev)
        bandE = torch.as_tensor(nE, device=self.dev)
        bandW = torch.as_tensor(w, device=self.dev)
        # template length per source from the band rule (Mc <= 1 M_sun), capped at 1024
        Ns = np.array([min(1024, wk.n_for_band(f, self.T, 1.0)) for f in self.src[:, 0]])
        th_all = torch.as_tensor(self.src, device=self.dev)
        for N in np.unique(Ns):
            sel = torch.as_tensor(np.nonzero(Ns == N)[0], device=self.dev)
            self._scatter((bandA, bandE), self.k_lo, th_all[sel].contiguous(), int(N), 1.0)
        # window copies
        gidx = torch.cat([torch.arange(k0 - self.k_lo, k0 - self.k_lo + N, device=self.dev)
                          for k0, N, _, _ in self.layout])
        self._gidx = gidx
        self._band0 = (bandA, bandE)
        self.dA = bandA[gidx].contiguous()
        self.dE = bandE[gidx].contiguous()
        self.wA = bandW[gidx].contiguous()
        self.wE = self.wA.clone()
        self.stats["synthesis_s"] = _sync(self.dev) - t0
        self.stats["sources"] = int(self.src.shape[0])
        self.stats["windows"] = self.n_win
        self.stats["window_bins"] = self.n_bins
        return self

    def windows(self, counts):
        """Descriptors (k0, W, N, data_off, cand_off, n) with counts[w] candidates in window w."""
        out, coff = [], 0
        for w, (k0, N, _, _) in enumerate(self.layout):
            out.append((k0, N, N, int(self.doff[w]), coff, int(counts[w])))
            coff += int(counts[w])
        return out

    def injected_snr(self):
        """Optimal SNR sqrt(<h|h>) of every injected source in the window that owns its f0."""
        kb = np.array([b for _, _, _, b in self.layout])
        owner = np.searchsorted(kb, self.src[:, 0] * self.T, side="right")
        owner = np.minimum(owner, self.n_win - 1)
        order = np.argsort(owner, kind="stable")
        counts = np.bincount(owner, minlength=self.n_win)
        th = torch.as_tensor(self.src[order], device=self.dev).contiguous()
        _, _, hh = self.ctx.loglik(self.windows(counts), self.dA, self.dE, self.wA, self.wE, th, prec=self.prec)
        snr = np.empty(self.src.shape[0])
        snr[order] = np.sqrt(np.maximum(hh.cpu().numpy(), 0.0))
        return snr, owner

    # -- search ------------------------------------------------------------

    def boxes(self):
        """Search boxes: Table 1's ranges with f0 over the padded segment, the
        segment's bins [ka, kb) widened by a quarter of its width on each side
        and kept inside the window."""
        b = np.empty((self.n_win, 16))
        for w, (k0, N, ka, kb) in enumerate(self.layout):
            lo, hi = _LO.copy(), _HI.copy()
            pad = 0.25 * (kb - ka)
            lo[0], hi[0] = max(ka - pad, k0) / self.T, min(kb + pad, k0 + N) / self.T
            hi[1] = float(wk.chirp_fdot(hi[0], 1.0))
            b[w] = np.concatenate([lo, hi])
        return b

    def _proposal_cov(self, win, theta, width=1.2 * math.sqrt(15.0)):
        """(n, 8, 8) covariances width^2 F^-1 from the observed Fisher matrix of
        the adjoint gradient (default: the T = 15 tempered width, widened by
        1.2), in natural units with eigenvalues floored and variances capped
        at the search box."""
        F = gbag.observed_fisher(self.ctx, win, self.dA, self.dE, self.wA, self.wE, theta, prec=self.prec)
        s = torch.ones_like(theta)
        s[:, 0] = 1.0 / self.T
        s[:, 1] = 1.0 / self.T ** 2
        s[:, 4] = theta[:, 4].abs()
        # 8x8 algebra on the host (no device linear-algebra library needed)
        s = s.cpu().numpy()
        Fs = F.cpu().numpy() * s[:, :, None] * s[:, None, :]
        ev, V = np.linalg.eigh(0.5 * (Fs + Fs.transpose(0, 2, 1)))
        ev = np.maximum(ev, 1e-8 * np.maximum(ev[:, -1:], 1e-300))
        C = (V / ev[:, None, :]) @ V.transpose(0, 2, 1) * width ** 2
        cap = np.array([4.0, 4.0, 1.0, 1.0, 1.0, 1.0, 1.0, 1.0]) ** 2
        d = np.sqrt(np.maximum(np.diagonal(C, axis1=1, axis2=2) / cap, 1.0))
        C = C / d[:, :, None] / d[:, None, :]
        return C * s[:, :, None] * s[:, None, :]

    def _wins(self, active, counts=None):
        """Descriptors of the windows `active` (counts[i] candidates for the i-th, default 0)."""
        out, coff = [], 0
        for i, w in enumerate(active):
            k0, N, _, _ = self.layout[w]
            c = 0 if counts is None else int(counts[i])
            out.append((k0, N, N, int(self.doff[w]), coff, c))
            coff += c
        return out

    def _refresh(self, active, bandA, bandE):
        """Window copies of the windows `active` from band arrays."""
        pos = torch.cat([torch.arange(int(self.doff[w]), int(self.doff[w]) + self.layout[w][1], device=self.dev)
                         for w in active])
        self.dA[pos] = bandA[self._gidx[pos]]
        self.dE[pos] = bandE[self._gidx[pos]]

    def _add_windows(self, ws, theta, sign):
        """Add sign * templates theta[i] to window ws[i]'s own copy."""
        for N in sorted({self.layout[w][1] for w in ws}):
            sel = [i for i, w in enumerate(ws) if self.layout[w][1] == N]
            th = torch.as_tensor(np.asarray(theta)[sel], device=self.dev).contiguous()
            for j0 in range(0, len(sel), 8192):
                part = [ws[i] for i in sel[j0:j0 + 8192]]
                hA, hE, q = self.ctx.waveform(th[j0:j0 + len(part)], N, "fp64")
                k0 = torch.as_tensor([self.layout[w][0] for w in part], device=self.dev)
                off = torch.as_tensor([int(self.doff[w]) for w in part], device=self.dev)
                loc = q[:, None] - N // 2 + torch.arange(N, device=self.dev)[None, :] - k0[:, None]
                ok = (loc >= 0) & (loc < N)
                idx = (loc + off[:, None])[ok]
                for tgt, h in ((self.dA, hA), (self.dE, hE)):
                    torch.view_as_real(tgt).index_add_(0, idx, sign * torch.view_as_real(h)[ok])

    def _subtract_windows(self, ws, theta):
        """Remove templates theta[i] from window ws[i]'s own copy."""
        self._add_windows(ws, theta, -1.0)

    def _joint_refit(self, ws, srcs, sweeps=2, iters=3):
        """Joint refinement of every source found in the windows ws (the
        step Alg. 2 takes with SLSQP after each new signal): maximising the
        multi-signal SNR of Eq. 11 over all the window's sources, amplitudes
        included, is maximising their joint likelihood, whose gradient for
        source k is the single-source gradient against the data minus the
        other sources.  So each sweep takes the sources slot by slot: add
        source k back to the (residual) window copy, which then holds
        d - sum_{j != k} s_j, polish it there, subtract the polished template.
        srcs: window -> list of theta, updated in place."""
        for _ in range(int(sweeps)):
            for k in range(max(len(srcs[w]) for w in ws)):
                wk_ = [w for w in ws if len(srcs[w]) > k]
                th = np.array([srcs[w][k] for w in wk_])
                self._add_windows(wk_, th, 1.0)
                pol, _ = gbag.newton_polish(self.ctx, self._wins(wk_), self.dA, self.dE, self.wA, self.wE,
                                            torch.as_tensor(th, device=self.dev).contiguous(), iters=iters,
                                            prec=self.prec)
                pol = pol.cpu().numpy()
                self._add_windows(wk_, pol, -1.0)
                for w, t in zip(wk_, pol):
                    srcs[w][k] = t.copy()

    def _subtract_band(self, bandA, bandE, found):
        """band -= templates of found (window, theta) pairs, each at its window's N."""
        for N in sorted({self.layout[w][1] for w, _ in found}):
            th = torch.as_tensor(np.array([t for w, t in found if self.layout[w][1] == N]), device=self.dev)
            self._scatter((bandA, bandE), self.k_lo, th.contiguous(), int(N), -1.0)

    def _posteriors(self, ws, best, boxes, n_post, post_batch, posterior, seed):
        acc_all = []
        for i in range(0, len(ws), post_batch):
            sub = list(ws[i:i + post_batch])
            win = self._wins(sub)
            mu = torch.as_tensor(best[i:i + len(sub)], device=self.dev).contiguous()
            if posterior == "kde":
                # the paper's proposals: uniform over the reduced box, then paired KDEs
                sig = np.sqrt(np.diagonal(self._proposal_cov(win, mu, width=1.0), axis1=1, axis2=2))
                box = reduced_box(best[i:i + len(sub)], sig, boxes[sub, :8], boxes[sub, 8:])
                ap = KDEPosterior(self.ctx, win, self.dA, self.dE, self.wA, self.wE, box, n=n_post,
                                  seed=seed + i, prec=self.prec).run()
                acc = ap.accepted.cpu().numpy()
            else:
                cov = self._proposal_cov(win, mu)
                ap = AnnealedPosterior(self.ctx, win, self.dA, self.dE, self.wA, self.wE, mu, cov, n=n_post,
                                       seed=seed + i, prec=self.prec).run()
                acc = ap.rounds.accepted.cpu().numpy()
            acc_all.extend(int(a) for a in acc)
            del ap
        return acc_all

    def _search_windows(self, active, n_rounds, tag, acc, boxes, pop, generations, snr_min, n_post, post_batch,
                        phase, posterior, noise, joint=True, polish_iters=6, seeds=None):
        """Search-and-subtract in the windows `active` (Alg. 2-3 per window):
        each round a genetic search over the padded segment in every active
        window and the polish; an optimum whose SNR on the window's residual
        (the data it was fitted to) passes the threshold has its template
        subtracted from the window's copy.  It is
        a source of the segment (theta_in) when its f0 lies in the unpadded
        segment, else a neighbour's signal spilling into the padding
        (theta_out), which stays subtracted but is not returned.  A window
        holding two or more sources of its own refits them jointly
        (_joint_refit) with theta_out held fixed; a window leaves the active
        set when a round finds nothing in it.  Then each source of the
        segment gets its posterior (Alg. 4) on the window's data minus every
        other found signal (the paper's d_posterior), at the final estimates.
        Returns [(window, theta, snr, accepted moves of its posterior)]."""
        active = np.asarray(active, dtype=int)
        srcs = {}
        orig = (self.dA.clone(), self.dE.clone())
        for r in range(n_rounds):
            if active.size == 0:
                break
            t0 = _sync(self.dev)
            wins = self._wins(active, [pop] * active.size)
            if noise == "median":   # the segment noise, updated after every subtraction
                self.ctx.noise_median(self._wins(active), self.dA, self.dE, debias=True, weights=(self.wA, self.wE))
            init = None
            if seeds is not None and len(seeds):
                # starting points from a shorter observation's search (Sec. III.E):
                # its signals whose f0 lies in the window's padded segment
                f = seeds[:, 0]
                init = [seeds[(f >= boxes[w, 0]) & (f < boxes[w, 8])] for w in active]
            ga = GASearch(self.ctx, wins, self.dA, self.dE, self.wA, self.wE, boxes[active], pop,
                          seed=self.seed + 17 * (r + 100 * tag), prec=self.prec, phase=phase, init=init)
            best = ga.run(generations, graph=True)
            del ga
            # gradient polish of every window's best
            allw = self._wins(active)
            th_b, _ = gbag.newton_polish(self.ctx, allw, self.dA, self.dE, self.wA, self.wE,
                                         torch.as_tensor(best, device=self.dev).contiguous(), iters=polish_iters,
                                         prec=self.prec)
            _, dh, hh = self.ctx.loglik(self._wins(active, [1] * active.size), self.dA, self.dE, self.wA, self.wE,
                                        th_b.contiguous(), prec=self.prec)
            best = th_b.cpu().numpy()
            snr = (dh / torch.sqrt(torch.clamp(hh, min=1e-300))).cpu().numpy()
            t1 = _sync(self.dev)
            acc["ga"] += t1 - t0
            acc["evals"] += pop * active.size * generations
            hit = np.nonzero(snr > snr_min)[0]
            if hit.size:
                ws = active[hit]
                self._subtract_windows(list(ws), best[hit])
                for w, i in zip(ws, hit):
                    _, _, ka, kb = self.layout[int(w)]
                    if ka <= best[i][0] * self.T < kb:
                        srcs.setdefault(int(w), []).append(best[i].copy())
                    else:
                        acc["out"] += 1
                t2 = _sync(self.dev)
                acc["sub"] += t2 - t1
                multi = [int(w) for w in ws if len(srcs.get(int(w), [])) > 1]
                if joint and multi:
                    self._joint_refit(multi, srcs)
                    acc["joint_s"] += _sync(self.dev) - t2
            active = active[hit]
        found = []
        if not srcs:
            return found
        ws_all = sorted(srcs)
        # Eq. 11 on the data the run started from: the SNR of the sum of each window's sources
        rho, _, _ = self.ctx.snr_multi(self._wins(ws_all, [len(srcs[w]) for w in ws_all]), orig[0], orig[1],
                                       self.wA, self.wE,
                                       torch.as_tensor(np.concatenate([np.array(srcs[w]) for w in ws_all]),
                                                       device=self.dev).contiguous())
        acc["joint_snr"].extend(float(x) for x in rho.cpu().numpy() if np.isfinite(x))
        acc["multi_windows"] += sum(1 for w in ws_all if len(srcs[w]) > 1)
        del orig
        # posteriors: slot by slot, source k of every window on d - sum_{j != k} s_j
        t3 = _sync(self.dev)
        for k in range(max(len(v) for v in srcs.values())):
            wk_ = [w for w in ws_all if len(srcs[w]) > k]
            th = np.array([srcs[w][k] for w in wk_])
            self._add_windows(wk_, th, 1.0)
            _, dh, hh = self.ctx.loglik(self._wins(wk_, [1] * len(wk_)), self.dA, self.dE, self.wA, self.wE,
                                        torch.as_tensor(th, device=self.dev).contiguous(), prec=self.prec)
            snr_k = (dh / torch.sqrt(torch.clamp(hh, min=1e-300))).cpu().numpy()
            pa = self._posteriors(np.array(wk_), th, boxes, n_post, post_batch, posterior,
                                  self.seed + 1000 * (k + 100 * tag)) if n_post > 0 else [0] * len(wk_)
            acc["n_post"] += len(pa)
            self._add_windows(wk_, th, -1.0)
            found.extend((w, th[i].copy(), float(snr_k[i]), a) for i, (w, a) in enumerate(zip(wk_, pa)))
        acc["post_s"] += _sync(self.dev) - t3
        return found

    def search(self, rounds=3, pop=1024, generations=100, snr_min=10.0, n_post=10000, post_batch=4096, phase=True,
               posterior="gauss", scheme="all", noise="true", joint=True, polish_iters=6, seeds=None):
        """Search every window for up to `rounds` signals.

        scheme="all": all windows at once on their own copies of the data.
        scheme="evenodd": the paper's three runs (Table 2, Alg. 3): the even
        segments for up to 3 signals on the data; the odd segments for up to
        `rounds` signals on the data minus the even runs' signals; the even
        segments again for up to `rounds` on the data minus the odd
        segments' signals, except those whose odd neighbours found nothing
        and that found fewer than 3 (their first-run signals are kept).
        noise="median": the weights of each searched window are its median
        periodogram (Sec. III.C), updated after every subtraction.
        joint: refit a window's sources jointly after each new one (Alg. 2)."""
        boxes = self.boxes()
        self.stats.update({"rounds": rounds, "pop": pop, "generations": generations, "snr_min": snr_min,
                           "proposals_per_posterior": n_post, "phase_maximised_fitness": phase,
                           "posterior_proposals": posterior, "scheme": scheme, "noise": noise,
                           "joint_refit": joint})
        wins = self.windows([pop] * self.n_win)
        th0 = torch.as_tensor(np.repeat(boxes[:, None, :8], pop, 1).reshape(-1, 8)
                              + np.repeat((boxes[:, None, 8:] - boxes[:, None, :8]) * 0.5, pop, 1).reshape(-1, 8),
                              device=self.dev).contiguous()
        self.stats["autotune"] = self.ctx.autotune(wins, self.dA, self.dE, self.wA, self.wE, th0, prec=self.prec,
                                                   reps=2)
        acc = {"ga": 0.0, "post_s": 0.0, "sub": 0.0, "joint_s": 0.0, "evals": 0, "n_post": 0, "joint_snr": [],
               "multi_windows": 0, "out": 0}
        kw = dict(boxes=boxes, pop=pop, generations=generations, snr_min=snr_min, n_post=n_post,
                  post_batch=post_batch, phase=phase, posterior=posterior, noise=noise, joint=joint,
                  polish_iters=polish_iters, seeds=None if seeds is None else np.asarray(seeds, dtype=np.float64))
        if scheme == "all":
            found = self._search_windows(np.arange(self.n_win), rounds, 0, acc, **kw)
        elif scheme == "evenodd":
            even, odd = np.arange(0, self.n_win, 2), np.arange(1, self.n_win, 2)
            run1 = self._search_windows(even, 3, 1, acc, **kw)
            t = _sync(self.dev)
            bA, bE = self._band0[0].clone(), self._band0[1].clone()
            self._subtract_band(bA, bE, [(f[0], f[1]) for f in run1])
            self._refresh(odd, bA, bE)
            acc["sub"] += _sync(self.dev) - t
            run2 = self._search_windows(odd, rounds, 2, acc, **kw)
            t = _sync(self.dev)
            n1 = np.bincount([f[0] for f in run1], minlength=self.n_win)
            n2 = np.bincount([f[0] for f in run2], minlength=self.n_win)
            redo = np.array([w for w in even if n1[w] >= 3 or (w > 0 and n2[w - 1] > 0) or
                             (w + 1 < self.n_win and n2[w + 1] > 0)], dtype=int)
            bA, bE = self._band0[0].clone(), self._band0[1].clone()
            self._subtract_band(bA, bE, [(f[0], f[1]) for f in run2])
            if redo.size:
                self._refresh(redo, bA, bE)
            acc["sub"] += _sync(self.dev) - t
            run3 = self._search_windows(redo, rounds, 3, acc, **kw)
            keep = set(int(w) for w in even) - set(int(w) for w in redo)
            found = run2 + run3 + [f for f in run1 if f[0] in keep]
            self.stats.update({"run_signals": [len(run1), len(run2), len(run3)], "even_searched_again": int(redo.size)})
        else:
            raise ValueError("scheme must be 'all' or 'evenodd'")
        self.found = [(0, w, th, s) for w, th, s, _ in found]
        post = [a for _, _, _, a in found]   # the catalogue's posteriors
        t_ga, evals = acc["ga"], acc["evals"]
        self.stats.update({"joint_refit_s": acc["joint_s"], "windows_with_several_sources": acc["multi_windows"],
                           "padding_signals_subtracted": acc["out"],
                           "joint_snr_median": float(np.median(acc["joint_snr"])) if acc["joint_snr"] else None})
        self.stats.update({"ga_s": t_ga, "posterior_s": acc["post_s"], "subtract_s": acc["sub"], "ga_evals": evals,
                           "ga_evals_per_s": evals / t_ga if t_ga > 0 else None, "recovered": len(found),
                           "posteriors": len(post), "posteriors_run": acc["n_post"],
                           "s_per_posterior": acc["post_s"] / acc["n_post"] if acc["n_post"] else None,
                           "median_accept_rate": float(np.median(post) / n_post) if post else None})
        return self.found

    def match(self, snr_inj, owner, n_near=4, batch=8192, snr_inj_search=None):
        """How the recoveries sit on the injections.  The paper's scores
        (Sec. IV): for every recovered source, the scaled error delta (Eq. 19)
        and the overlap O (Eq. 20) against each of the n_near injected sources
        nearest in frequency, from the 2 x 2 Gram matrices of gb_snr_multi
        (templates of the recovered source's window length N over 2N bins
        centred on its carrier, weights 1/S of the analytic PSD); the pair
        with the smallest delta is its match.  Reported: the fractions of
        recoveries with delta < 0.3 and with O > 0.9, the injected sources
        above the SNR threshold and how many distinct ones are matched with
        delta < 0.3; also the fractions within one and three frequency bins
        and the median ratio of recovered to that injection's optimal SNR
        (snr_inj_search: the injected SNRs under the weights the search used,
        when they differ from the instrument's, so that both SNRs of the
        ratio see the same noise; snr_inj counts the loud injections)."""
        f_inj = self.src[:, 0]
        snr_ref = snr_inj if snr_inj_search is None else snr_inj_search
        order = np.argsort(f_inj)
        fs = f_inj[order]
        d, ratio = [], []
        for _, w, th, s in self.found:
            i = np.clip(np.searchsorted(fs, th[0]), 1, fs.size - 1)
            j = order[i - 1] if abs(fs[i - 1] - th[0]) < abs(fs[i] - th[0]) else order[i]
            d.append(abs(f_inj[j] - th[0]) * self.T)
            ratio.append(s / max(snr_ref[j], 1e-300))
        d = np.array(d)
        loud = int(np.sum(snr_inj > self.stats.get("snr_min", 10.0)))
        out = {"within_1_bin": float(np.mean(d < 1.0)) if d.size else None,
               "within_3_bins": float(np.mean(d < 3.0)) if d.size else None,
               "median_snr_ratio": float(np.median(ratio)) if ratio else None,
               "injected_above_threshold": loud, "recovered_over_loud": len(self.found) / max(1, loud)}
        if not self.found:
            return out
        # delta and O against the nearest injections
        rec = np.array([th for _, _, th, _ in self.found])
        Ns = np.array([self.layout[w][1] for _, w, _, _ in self.found])
        pos = np.searchsorted(fs, rec[:, 0])
        cand = np.clip(pos[:, None] + np.arange(-n_near // 2, n_near - n_near // 2)[None, :], 0, fs.size - 1)
        inj = order[cand]                                                # (n_rec, n_near)
        n_rec = rec.shape[0]
        best_d = np.full(n_rec, np.inf)
        best_o = np.full(n_rec, -np.inf)
        best_j = np.full(n_rec, -1)
        pairs = [(r, k) for r in range(n_rec) for k in range(n_near)]
        for b0 in range(0, len(pairs), batch):
            part = pairs[b0:b0 + batch]
            wins, th, wts, off = [], [], [], 0
            for i, (r, k) in enumerate(part):
                N = int(Ns[r])
                q = int(math.floor((rec[r, 0] + 0.5 * rec[r, 1] * self.T) * self.T + 0.5))
                k0 = q - N
                wins.append((k0, 2 * N, N, off, 2 * i, 2))
                wts.append(1.0 / wk.psd_AE(np.maximum(np.arange(k0, k0 + 2 * N), 1) / self.T))
                th += [rec[r], self.src[inj[r, k]]]
                off += 2 * N
            wA = torch.as_tensor(np.concatenate(wts), device=self.dev)
            _, G, _ = self.ctx.snr_multi(wins, None, None, wA, wA, torch.as_tensor(np.array(th), device=self.dev),
                                         kmax=2)
            G = G.cpu().numpy()
            rr, ri, ii = G[:, 0, 0], G[:, 0, 1], G[:, 1, 1]
            with np.errstate(invalid="ignore", divide="ignore"):   # an injection with no bin in the window
                dl = np.nan_to_num((rr - 2 * ri + ii) / rr, nan=np.inf)
                ov = np.nan_to_num(ri / np.sqrt(rr * ii), nan=-np.inf)
            for i, (r, k) in enumerate(part):
                if dl[i] < best_d[r]:
                    best_d[r], best_j[r] = dl[i], inj[r, k]
                best_o[r] = max(best_o[r], ov[i])
        good = best_d < 0.3
        by_band = {}
        for lo, hi in ((0.0, 2e-3), (2e-3, 5e-3), (5e-3, 10e-3), (10e-3, None)):
            m = (rec[:, 0] >= lo) & ((rec[:, 0] < hi) if hi is not None else True)
            if m.any():
                by_band["%g-%s mHz" % (lo * 1e3, "%g" % (hi * 1e3) if hi is not None else "")] = {
                    "recovered": int(m.sum()), "delta_lt_0.3": float(np.mean(good[m]))}
        out.update({"delta_lt_0.3": float(np.mean(good)), "overlap_gt_0.9": float(np.mean(best_o > 0.9)),
                    "delta_lt_0.3_by_band": by_band,
                    "median_delta": float(np.median(best_d)),
                    "matched_injected_delta_lt_0.3": int(np.unique(best_j[good]).size),
                    "matched_over_loud": float(np.unique(best_j[good]).size / max(1, loud)),
                    "match_metric": "delta (Eq. 19) and overlap (Eq. 20) against the %d injections nearest in "
                                    "frequency; delta < 0.3 counts as matched" % n_near})
        return out


def run(ctx, n_src=200000, f_lo=0.3e-3, f_hi=15e-3, T=2 * wk.YEAR, rounds=3, pop=1024, generations=100,
        snr_min=10.0, n_post=10000, seed=wk.SEED_BASE + 5, warm=True, phase=True, posterior="gauss", scheme="all",
        noise="true", joint=True, amp="loguniform", polish_iters=6, t_short=None):
    """Config 5 end to end; returns the statistics (wall times in seconds).
    warm: run a small instance first, so that one-time library initialisation
    (kernel modules, solver handles) is not in the times.  amp: the
    population's amplitude law (workloads.fullband_sources).  t_short: if
    given, the same sources observed for t_short seconds are searched first
    (own context, own noise, no posteriors) and their signals start the
    searches of the full observation in their windows (Sec. III.E); a
    sequence of durations is a ladder, each stage seeded by the one before
    (the paper's 0.5, 1 and 2 yr)."""
    if warm:
        small = FullBand(ctx, wk.fullband_sources(200, 2e-3, 2.1e-3, seed + 1), wk.fullband_layout(2e-3, 2.1e-3, T),
                         T, seed=seed + 1).synthesize()
        small.injected_snr()
        small.search(rounds=1, pop=64, generations=4, snr_min=snr_min, n_post=256, posterior=posterior,
                     scheme=scheme, noise=noise, joint=joint)
    t0 = _sync(ctx.device)
    sources = wk.fullband_sources(n_src, f_lo, f_hi, seed, amp=amp)
    seeds, short = None, {}
    ladder = [] if t_short is None else sorted(float(x) for x in np.atleast_1d(t_short) if float(x) > 0)
    for k, ts in enumerate(ladder):
        # Sec. III.E: search the same sources observed for ts first (its own
        # context, noise and windows, no posteriors); its signals start the
        # searches of the next, longer observation in their windows
        ctx_s = api.Context(ts, arm_L=ctx.arm_L, device=ctx.device.index)
        fs = FullBand(ctx_s, sources, wk.fullband_layout(f_lo, f_hi, ts), ts, seed=seed + 7 + k).synthesize()
        fs.search(rounds=rounds, pop=pop, generations=generations, snr_min=snr_min, n_post=0, phase=phase,
                  scheme=scheme, noise=noise, joint=joint, polish_iters=polish_iters, seeds=seeds)
        seeds = np.array([th for _, _, th, _ in fs.found]) if fs.found else np.zeros((0, 8))
        short.setdefault("t_short_yr", []).append(ts / wk.YEAR)
        short.setdefault("short_recovered", []).append(len(fs.found))
        del fs
        ctx_s.close()
    if ladder:
        short["short_wall_s"] = _sync(ctx.device) - t0
    fb = FullBand(ctx, sources, wk.fullband_layout(f_lo, f_hi, T), T, seed=seed).synthesize()
    snr_inj, owner = fb.injected_snr()
    fb.search(rounds=rounds, pop=pop, generations=generations, snr_min=snr_min, n_post=n_post, phase=phase,
              posterior=posterior, scheme=scheme, noise=noise, joint=joint, polish_iters=polish_iters, seeds=seeds)
    st = dict(fb.stats)
    st.update(short)
    # with median-noise weights the recovered SNRs are measured against the
    # segments' estimated PSD: compare them with the injections' SNRs under
    # the same weights (the instrument-PSD SNRs still count the loud ones)
    snr_search = fb.injected_snr()[0] if noise == "median" else None
    st.update(fb.match(snr_inj, owner, snr_inj_search=snr_search))
    st["wall_s"] = _sync(ctx.device) - t0
    st["search_wall_s"] = st["ga_s"] + st["posterior_s"] + st["subtract_s"] + st["joint_refit_s"]
    return st
