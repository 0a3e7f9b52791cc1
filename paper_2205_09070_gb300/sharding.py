"""Host-side logic for running independent GPs on several GPUs.

The hot path does not shard one GP (one matrix, one GPU); what shards is a
batch of independent instances (each a full GP of its own): instances are
split across ranks with no collective on the data path, each rank evaluates
its share through the C ABI, and results are gathered once at the end.  The
benchmark runs one replica per rank and reports the max over ranks of the
timed region.
"""

from __future__ import annotations

import numpy as np


def shard_instances(offsets, world: int, rank: int) -> np.ndarray:
    """Indices of the instances rank `rank` evaluates.  Instances are dealt in
    decreasing size to the rank with the least work so far (ties: lower
    rank), which balances total points; the result is sorted."""
    offsets = np.asarray(offsets, dtype=np.int64)
    sizes = np.diff(offsets)
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad world size / rank")
    load = np.zeros(world, dtype=np.int64)
    owner = np.empty(len(sizes), dtype=np.int64)
    for k in sorted(range(len(sizes)), key=lambda q: (-int(sizes[q]), q)):
        r = int(np.argmin(load))
        owner[k] = r
        load[r] += max(int(sizes[k]), 1)
    return np.nonzero(owner == rank)[0]


def local_offsets(offsets, idx) -> tuple[np.ndarray, np.ndarray]:
    """Offsets of the selected instances packed contiguously, and the gather
    index of their points in the original arrays."""
    offsets = np.asarray(offsets, dtype=np.int64)
    sizes = offsets[np.asarray(idx) + 1] - offsets[np.asarray(idx)]
    lo = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    pts = np.concatenate([np.arange(offsets[k], offsets[k + 1]) for k in idx]) if len(idx) else np.zeros(0, np.int64)
    return lo, pts


def gather_results(idx_local, lml_local, grad_local, n_inst: int, n_params: int, group=None):
    """Assemble every rank's (instance index, lml, grad) into full arrays on
    all ranks (torch.distributed all_gather_object; called once, after the
    evaluations)."""
    import torch.distributed as dist
    mine = (list(map(int, idx_local)), np.asarray(lml_local).tolist(), np.asarray(grad_local).tolist())
    world = dist.get_world_size(group)
    parts = [None] * world
    dist.all_gather_object(parts, mine, group=group)
    lml = np.full(n_inst, np.nan)
    grad = np.full((n_inst, n_params), np.nan)
    for idx, lv, gv in parts:
        for q, k in enumerate(idx):
            lml[k] = lv[q]
            grad[k] = gv[q]
    return lml, grad


def max_over_ranks(value: float, device=None, group=None) -> float:
    """Max of a per-rank scalar (timed-region milliseconds) over all ranks."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
