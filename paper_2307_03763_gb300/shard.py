"""Window sharding across ranks (one process per GPU).

Frequency windows are independent problems (Sec. III.E analyses non-adjacent
segments in parallel), so a multi-GPU run gives each rank a disjoint set of
windows and needs no exchange on the data path: each rank evaluates its
windows with its own library context, and the only collective is the final
gather of per-candidate results.  Windows are assigned greedily, most
expensive first, to the least-loaded rank (cost ~ n_cand N (log2 N + 12)).
This module only computes index layouts and moves results; it does no
likelihood arithmetic.
"""
import math

import numpy as np


def window_cost(window):
    k0, W, N, doff, coff, nc = window
    return float(nc) * N * (math.log2(N) + 12.0)


def assign(windows, world):
    """Rank of every window (longest-processing-time-first greedy)."""
    order = sorted(range(len(windows)), key=lambda i: -window_cost(windows[i]))
    load = [0.0] * world
    owner = [0] * len(windows)
    for i in order:
        r = min(range(world), key=lambda j: (load[j], j))
        owner[i] = r
        load[r] += window_cost(windows[i])
    return owner


class Shard:
    """The part of a workload one rank evaluates, re-laid out compactly.

    windows: the rank's windows with data_off and cand_off rebased into the
    rank's own arrays; data_index / cand_index map those arrays back to the
    global bins and candidate rows.
    """

    def __init__(self, windows, world, rank):
        owner = assign(windows, world)
        self.window_ids = [i for i in range(len(windows)) if owner[i] == rank]
        self.windows = []
        data_index, cand_index = [], []
        doff = coff = 0
        for i in self.window_ids:
            k0, W, N, d0, c0, nc = windows[i]
            self.windows.append((k0, W, N, doff, coff, nc))
            data_index.append(np.arange(d0, d0 + W))
            cand_index.append(np.arange(c0, c0 + nc))
            doff += W
            coff += nc
        self.data_index = np.concatenate(data_index) if data_index else np.zeros(0, np.int64)
        self.cand_index = np.concatenate(cand_index) if cand_index else np.zeros(0, np.int64)

    def take_data(self, *arrays):
        return tuple(a[self.data_index] for a in arrays)

    def take_candidates(self, theta):
        return theta[self.cand_index]


def gather(values, shard, n_total, group=None):
    """Scatter every rank's per-candidate results into one (n_total, ...) array
    on every rank (torch.distributed all_gather of the local slices)."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    vals = torch.as_tensor(values)
    idx = torch.as_tensor(shard.cand_index, dtype=torch.int64, device=vals.device)
    n_local = torch.tensor([vals.shape[0]], dtype=torch.int64, device=vals.device)
    sizes = [torch.zeros_like(n_local) for _ in range(world)]
    dist.all_gather(sizes, n_local, group=group)
    m = int(max(int(s.item()) for s in sizes))
    pad_v = torch.zeros((m,) + tuple(vals.shape[1:]), dtype=vals.dtype, device=vals.device)
    pad_i = torch.full((m,), -1, dtype=torch.int64, device=vals.device)
    pad_v[:vals.shape[0]] = vals
    pad_i[:idx.shape[0]] = idx
    all_v = [torch.zeros_like(pad_v) for _ in range(world)]
    all_i = [torch.zeros_like(pad_i) for _ in range(world)]
    dist.all_gather(all_v, pad_v, group=group)
    dist.all_gather(all_i, pad_i, group=group)
    out = torch.zeros((n_total,) + tuple(vals.shape[1:]), dtype=vals.dtype, device=vals.device)
    for v, i in zip(all_v, all_i):
        keep = i >= 0
        out[i[keep]] = v[keep]
    return out
