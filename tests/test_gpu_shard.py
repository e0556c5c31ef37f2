"""Window sharding with the CUDA library on every rank.

Two processes (gloo for the gather; both on cuda:0 -- their kernels never wait
on one another) each evaluate their share of the windows (shard.Shard, the
cost-balanced assignment) with gb_loglik and gb_mh_certified; shard.gather
puts the per-candidate results back together.  The gathered logL (FP64 and
mixed) and the certified chains must equal one process's evaluation of all
windows bit for bit: every candidate and chain is computed by the same code
whichever rank holds it.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

pytestmark = pytest.mark.gpu


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _workload():
    from paper_2307_03763_gb300 import workloads as wk
    from tests import _data
    wl = wk.band_windows(n_win=10, cand_range=(300, 300), seed=wk.SEED_BASE + 92, T=2 * wk.YEAR)
    dA, dE = _data.inject(wl)
    rng = np.random.default_rng(7)
    log_g = rng.normal(0.0, 1.0, wl.n_cand)
    return wl, dA, dE, log_g


def _evaluate(api, wl, windows, dA, dE, wA, wE, theta, log_g, log_u, dev):
    """logL (FP64, mixed) and certified chains of the given windows."""
    c = lambda x, dt: torch.as_tensor(np.ascontiguousarray(x)).to(dev, dt)
    ctx = api.Context(wl.T, device=dev.index)
    args = (c(dA, torch.complex128), c(dE, torch.complex128), c(wA, torch.float64), c(wE, torch.float64),
            c(theta, torch.float64))
    l64 = ctx.loglik(windows, *args, prec="fp64")[0].cpu()
    lmx = ctx.loglik(windows, *args, prec="mixed")[0].cpu()
    nw, n = len(windows), windows[0][5]
    temp = torch.full((nw,), 3.0, dtype=torch.float64, device=dev)
    out = ctx.mh_certified(windows, *args, c(log_g.reshape(nw, n), torch.float64),
                           c(log_u.reshape(nw, n), torch.float64), temp)
    chain, pending = out[0].cpu(), int(out[6].item())
    ctx.close()
    return l64, lmx, chain, pending


def _rank(rank, world, port, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2307_03763_gb300 import api
        from paper_2307_03763_gb300 import shard as sh
        dev = torch.device("cuda", 0)
        torch.cuda.set_device(dev)
        wl, dA, dE, log_g = _workload()
        s = sh.Shard(wl.windows, world, rank)
        d = s.take_data(dA, dE, wl.w_A, wl.w_E)
        l64, lmx, chain, pending = _evaluate(api, wl, s.windows, *d, s.take_candidates(wl.theta),
                                             s.take_candidates(log_g), s.take_candidates(wl.log_u), dev)
        # chain entries are local proposal indices within each window: the same
        # numbers a single process writes, so they gather like any per-row value
        g64 = sh.gather(l64, s, wl.n_cand)
        gmx = sh.gather(lmx, s, wl.n_cand)
        gch = sh.gather(chain.reshape(-1), s, wl.n_cand)
        pend = torch.tensor([pending])
        dist.all_reduce(pend)
        if rank == 0:
            torch.save({"l64": g64, "lmx": gmx, "chain": gch, "pending": int(pend), "windows": s.window_ids},
                       out_path)
    finally:
        dist.destroy_process_group()


def test_sharded_library_evaluation_equals_single_process(tmp_path):
    from paper_2307_03763_gb300 import api, build
    build.build()
    out = str(tmp_path / "r0.pt")
    mp.start_processes(_rank, args=(2, _free_port(), out), nprocs=2, start_method="spawn", join=True)
    res = torch.load(out)
    wl, dA, dE, log_g = _workload()
    dev = torch.device("cuda", 0)
    l64, lmx, chain, pending = _evaluate(api, wl, wl.windows, dA, dE, wl.w_A, wl.w_E, wl.theta, log_g, wl.log_u,
                                         dev)
    assert res["pending"] == 0 and pending == 0
    assert 0 < len(res["windows"]) < len(wl.windows)          # rank 0 holds a strict part
    assert torch.equal(res["l64"], l64)
    assert torch.equal(res["lmx"], lmx)
    assert torch.equal(res["chain"], chain.reshape(-1))
