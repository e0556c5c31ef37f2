"""Multi-rank window sharding on CPU ranks (gloo, world size 2).

Each rank takes its windows from the LPT assignment, evaluates them with the
FP64 oracle (the CUDA library needs a GPU; the host logic is what is under
test here) and the per-candidate results are gathered.  The gathered logL
must equal a single-process evaluation of all windows, every window must be
owned by exactly one rank, and the cost must be balanced.
"""
import os
import socket

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2307_03763_gb300 import shard as sh
from paper_2307_03763_gb300 import workloads as wk


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _workload():
    return wk.band_windows(n_win=9, cand_range=(3, 7), seed=wk.SEED_BASE + 90)


def _rank(rank, world, port, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import gb as ogb
        wl = _workload()
        s = sh.Shard(wl.windows, world, rank)
        nA, nE, wA, wE = s.take_data(wl.noise_A, wl.noise_E, wl.w_A, wl.w_E)
        th = s.take_candidates(wl.theta)
        logL, _, _ = ogb.loglik(s.windows, nA, nE, wA, wE, th, wl.T)
        full = sh.gather(logL, s, wl.n_cand)
        owned = torch.zeros(len(wl.windows), dtype=torch.int64)
        owned[s.window_ids] = 1
        dist.all_reduce(owned)
        if rank == 0:
            torch.save({"logL": full, "owned": owned}, out_path)
    finally:
        dist.destroy_process_group()


def test_sharded_evaluation_equals_single_process(tmp_path):
    from oracle import gb as ogb
    out = str(tmp_path / "r0.pt")
    mp.start_processes(_rank, args=(2, _free_port(), out), nprocs=2, start_method="spawn", join=True)
    res = torch.load(out)
    wl = _workload()
    ref, _, _ = ogb.loglik(wl.windows, wl.noise_A, wl.noise_E, wl.w_A, wl.w_E, wl.theta, wl.T)
    assert torch.equal(res["owned"], torch.ones(len(wl.windows), dtype=torch.int64))
    assert torch.allclose(res["logL"], ref, rtol=1e-12, atol=0)


def test_assignment_balances_cost():
    wl = wk.band_windows(n_win=64, cand_range=(100, 2000), seed=wk.SEED_BASE + 91)
    for world in (2, 4, 8):
        owner = sh.assign(wl.windows, world)
        load = np.zeros(world)
        for w, r in zip(wl.windows, owner):
            load[r] += sh.window_cost(w)
        biggest = max(sh.window_cost(w) for w in wl.windows)
        assert load.max() - load.min() <= biggest + 1e-9
