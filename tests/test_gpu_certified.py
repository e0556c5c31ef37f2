"""Chains from mixed-precision likelihoods that equal the FP64 chains (Alg. 4, Eq. 13).

gb_mh_certified evaluates every proposal in mixed precision, builds the
independence MH chains, and re-evaluates in FP64 (gb_loglik_rows) exactly the
proposals whose accept/reject decision the mixed error bound cannot settle.
The bars here are exact: chain indices and acceptance counts equal to those of
gb_loglik (FP64) followed by gb_mh_independence, re-evaluated rows equal to the
FP64 path bit for bit, the other rows equal to the mixed path bit for bit.  The
FP64 path itself is checked against the oracle to 1e-10 in test_gpu_parity.py.
"""
import numpy as np
import pytest
import torch

from paper_2307_03763_gb300 import workloads as wk
from tests import _data

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _cuda(x, dtype):
    return torch.as_tensor(np.ascontiguousarray(x)).to(device=DEV, dtype=dtype)


@pytest.fixture(scope="module")
def api():
    from paper_2307_03763_gb300 import api, build
    build.build()
    return api


@pytest.fixture(scope="module")
def posterior(api):
    """The 16-window, 10,000-proposal workload: SNR 20-200 sources, proposals
    from a Gaussian of 10 Fisher widths around each (oracle templates)."""
    wl = wk.posterior_windows()
    rng = np.random.default_rng(5)
    srcs, snr = [], []
    th = np.empty((wl.n_cand, 8))
    lg = np.empty(wl.n_cand)
    for w, (k0, W, N, doff, coff, nc) in enumerate(wl.windows):
        s = wl.sources[w][0].copy()
        s[4] = wl.meta["snr"][w] / _data.unit_snr(s, wl.windows[w], wl.w_A, wl.w_E, wl.T)
        srcs.append([s])
        sig = _data.fisher_sigma(s, wl.windows[w], wl.w_A, wl.w_E, wl.T)
        th[coff:coff + nc], lg[coff:coff + nc] = wk.gaussian_proposals(s, 10 * sig, nc, rng)
    dA, dE = _data.inject(wl, srcs)
    ctx = api.Context(wl.T)
    args = (_cuda(dA, torch.complex128), _cuda(dE, torch.complex128), _cuda(wl.w_A, torch.float64),
            _cuda(wl.w_E, torch.float64), _cuda(th, torch.float64))
    nw, n = len(wl.windows), wl.windows[0][5]
    yield dict(wl=wl, ctx=ctx, args=args, nw=nw, n=n, log_g=_cuda(lg.reshape(nw, n), torch.float64),
               log_u=_cuda(wl.log_u.reshape(nw, n), torch.float64), snr=np.asarray(wl.meta["snr"]))
    ctx.close()


def _fp64_chain(P, log_u, temp, literal=False):
    ctx, wl = P["ctx"], P["wl"]
    l64 = ctx.loglik(wl.windows, *P["args"], prec="fp64")[0]
    ch, acc = ctx.mh_independence(l64.view(P["nw"], P["n"]), P["log_g"], log_u, temp, literal=literal)
    return l64, ch, acc


def _check_certified(P, api, log_u, temp, literal=False, max_iter=3):
    ctx, wl = P["ctx"], P["wl"]
    l64, ch64, acc64 = _fp64_chain(P, log_u, temp, literal)
    lmx = ctx.loglik(wl.windows, *P["args"], prec="mixed")[0]
    ch, acc, logL, dh, hh, n_exact, pending = ctx.mh_certified(wl.windows, *P["args"], P["log_g"], log_u, temp,
                                                               literal=literal, max_iter=max_iter)
    torch.cuda.synchronize()
    assert int(pending.item()) == 0
    assert torch.equal(ch, ch64)
    assert torch.equal(acc, acc64)
    # re-evaluated rows carry the FP64 path's bits, the others the mixed path's
    redo = logL != lmx
    assert torch.equal(logL[redo], l64[redo])
    assert torch.equal(logL[~redo], lmx[~redo])
    assert int(redo.sum()) <= int(n_exact.sum())
    return ch, ch64, lmx, l64, int(n_exact.sum())


@pytest.mark.parametrize("temp_value,literal", [(1.0, False), (15.0, False), (3.0, True)])
def test_certified_chains_equal_fp64_chains(api, posterior, temp_value, literal):
    P = posterior
    temp = torch.full((P["nw"],), temp_value, dtype=torch.float64, device=DEV)
    ch, ch64, lmx, l64, n_exact = _check_certified(P, api, P["log_u"], temp, literal)
    # a few proposals per chain at most are re-evaluated
    assert n_exact <= 0.05 * P["nw"] * P["n"], n_exact


def _adversarial_log_u(l64, log_g, log_u, temp, frac, rng):
    """log u_i placed one ulp either side of the FP64 decision threshold Delta_i
    (tempered form, w = logL/T - log g) on a fraction of the steps, walking the
    FP64 chain: those decisions flip under any error of the likelihood."""
    L, G, U = l64.cpu().numpy(), log_g.cpu().numpy(), log_u.cpu().numpy().copy()
    Tv = temp.cpu().numpy()
    nw, n = G.shape
    for r in range(nw):
        T = Tv[r]
        w = (L[r] / T - G[r]) if T != 1.0 else (L[r] - G[r])
        c = 0
        for i in range(1, n):
            d = w[i] - w[c]
            if -30.0 < d < 0.0 and rng.random() < frac:
                U[r, i] = np.nextafter(d, -np.inf) if rng.random() < 0.5 else np.nextafter(d, np.inf)
            if U[r, i] < min(0.0, d):
                c = i
    return torch.as_tensor(U).to(DEV)


@pytest.mark.parametrize("temp_value", [1.0, 5.0])
def test_certified_chains_at_adversarial_thresholds(api, posterior, temp_value):
    # decisions on a knife edge: the chain from the mixed values alone takes
    # other paths, the certified chain still equals the FP64 chain
    P = posterior
    rng = np.random.default_rng(17)
    temp = torch.full((P["nw"],), temp_value, dtype=torch.float64, device=DEV)
    l64, _, _ = _fp64_chain(P, P["log_u"], temp)
    lu = _adversarial_log_u(l64.view(P["nw"], P["n"]), P["log_g"], P["log_u"], temp, 0.05, rng)
    ch, ch64, lmx, _, n_exact = _check_certified(P, api, lu, temp, max_iter=8)
    plain, _ = P["ctx"].mh_independence(lmx.view(P["nw"], P["n"]), P["log_g"], lu, temp)
    assert not torch.equal(plain, ch64)          # the mixed values alone decide otherwise
    assert n_exact > 0


def test_certified_pending_reports_unfinished_passes(api, posterior):
    # with one pass on the adversarial inputs the queue is not empty: pending > 0
    P = posterior
    rng = np.random.default_rng(18)
    temp = torch.ones(P["nw"], dtype=torch.float64, device=DEV)
    l64, _, _ = _fp64_chain(P, P["log_u"], temp)
    lu = _adversarial_log_u(l64.view(P["nw"], P["n"]), P["log_g"], P["log_u"], temp, 0.2, rng)
    out = P["ctx"].mh_certified(P["wl"].windows, *P["args"], P["log_g"], lu, temp, max_iter=1)
    torch.cuda.synchronize()
    assert int(out[6].item()) > 0


def test_certified_empty_chains_report_nothing_pending(api, posterior):
    # windows of zero proposals: no chain to build, so pending and the
    # re-evaluation counts are written as zero (not left as they were)
    P = posterior
    dA, dE, wA, wE, _ = P["args"]
    wins = [(k0, W, N, doff, 0, 0) for (k0, W, N, doff, coff, nc) in P["wl"].windows[:3]]
    theta = torch.empty((0, 8), dtype=torch.float64, device=DEV)
    z = torch.empty((3, 0), dtype=torch.float64, device=DEV)
    temp = torch.ones(3, dtype=torch.float64, device=DEV)
    e = lambda: torch.empty(0, dtype=torch.float64, device=DEV)
    n_exact = torch.full((3,), -7, dtype=torch.int32, device=DEV)
    pending = torch.full((1,), -7, dtype=torch.int32, device=DEV)
    out = (torch.empty((3, 0), dtype=torch.int32, device=DEV), torch.zeros(3, dtype=torch.int32, device=DEV),
           e(), e(), e(), n_exact, pending)
    P["ctx"].mh_certified(wins, dA, dE, wA, wE, theta, z, z, temp, out=out)
    torch.cuda.synchronize()
    assert int(pending.item()) == 0
    assert torch.equal(n_exact, torch.zeros(3, dtype=torch.int32, device=DEV))


def test_loglik_rows_bit_identical_to_loglik(api):
    # ragged windows of every N; listed subsets, partial ranges, entries of
    # another window (skipped), empty lists; unlisted rows untouched
    wl = wk.band_windows(seed=wk.SEED_BASE + 41, n_win=14, cand_range=(30, 80))
    ctx = api.Context(wl.T)
    dA, dE = _data.inject(wl)
    args = (_cuda(dA, torch.complex128), _cuda(dE, torch.complex128), _cuda(wl.w_A, torch.float64),
            _cuda(wl.w_E, torch.float64), _cuda(wl.theta, torch.float64))
    ref = [x.clone() for x in ctx.loglik(wl.windows, *args, prec="fp64")]
    rng = np.random.default_rng(3)
    n = wl.theta.shape[0]
    rows = np.full(n, -1, np.int32)
    lo, hi = np.zeros(len(wl.windows), np.int32), np.zeros(len(wl.windows), np.int32)
    expect = np.zeros(n, bool)
    for w, (k0, W, N, doff, coff, nc) in enumerate(wl.windows):
        perm = coff + rng.permutation(nc)
        rows[coff:coff + nc] = perm
        if w % 5 == 4:
            continue                                    # empty list
        a = int(rng.integers(0, nc // 2))
        b = int(rng.integers(a, nc + 1))
        lo[w], hi[w] = a, b
        if w == 0:
            hi[w] = nc + 1000                           # clamped to n_cand
        if w % 5 == 3 and b > a:
            rows[coff + a] = 0 if coff > 0 else n - 1   # another window's row: skipped
        expect[[r for r in rows[coff + a:coff + min(int(hi[w]), nc)] if coff <= r < coff + nc]] = True
    sentinel = -12345.0
    out = tuple(torch.full((n,), sentinel, dtype=torch.float64, device=DEV) for _ in range(3))
    ctx.loglik_rows(wl.windows, *args, _cuda(rows, torch.int32), _cuda(lo, torch.int32), _cuda(hi, torch.int32),
                    out=out)
    e = torch.as_tensor(expect).to(DEV)
    for o, r in zip(out, ref):
        assert torch.equal(o[e], r[e])
        assert bool((o[~e] == sentinel).all())
    assert int(e.sum()) > 100
    ctx.close()
