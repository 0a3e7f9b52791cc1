"""Multi-rank host logic on CPU (gloo, world size 2): instance sharding for
batches of independent GPs, result gathering, and the max-over-ranks timing
the benchmark reports.  No GPU is used."""

import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2205_09070_gb300 import sharding as S
from paper_2205_09070_gb300 import workloads as W


def test_shards_cover_every_instance_once_and_balance():
    probs = W.batch_2d(seed=4, n_inst=256)
    offsets = np.concatenate([[0], np.cumsum([q.n for q in probs])])
    for world in (1, 2, 3, 8):
        parts = [S.shard_instances(offsets, world, r) for r in range(world)]
        allk = np.sort(np.concatenate(parts))
        assert np.array_equal(allk, np.arange(256))
        loads = [int(np.sum(np.diff(offsets)[p])) for p in parts]
        assert max(loads) - min(loads) <= max(np.diff(offsets))     # greedy bound
    lo, pts = S.local_offsets(offsets, np.array([3, 7]))
    assert lo[-1] == len(pts) == (offsets[4] - offsets[3]) + (offsets[8] - offsets[7])
    assert pts[0] == offsets[3] and pts[-1] == offsets[8] - 1


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        n_inst, n_params = 10, 3
        offsets = np.arange(0, 11) * 5
        idx = S.shard_instances(offsets, world, rank)
        # stand-in per-instance results: lml = k, grad = (k, 2k, 3k)
        lml = idx.astype(float)
        grad = np.stack([idx * 1.0, idx * 2.0, idx * 3.0], axis=1) if len(idx) else np.zeros((0, 3))
        L, Gr = S.gather_results(idx, lml, grad, n_inst, n_params)
        t = S.max_over_ranks(10.0 + rank)
        out.put((rank, L.tolist(), Gr.tolist(), t))
    finally:
        dist.destroy_process_group()


def test_gloo_two_ranks_gather_and_max():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, L, Gr, t in res:
        assert L == list(map(float, range(10)))
        assert np.array_equal(np.array(Gr), np.stack([np.arange(10), 2 * np.arange(10), 3 * np.arange(10)], 1))
        assert t == 11.0
