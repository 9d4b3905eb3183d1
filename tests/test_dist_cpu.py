"""Multi-GPU host logic on CPU ranks (gloo, world size 2): replicas only.

The walk shards over walkers with no data-path collective; bench.py runs one
replica per GPU.  These checks cover what the replicas rely on: every rank
builds the identical graph and update batches from the seeds, walker seeds
differ by rank, and the timing reductions (max over ranks) and step sums.
"""
import hashlib
import os
import socket

import numpy as np
import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import sys

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    import workloads as W

    wl = W.make_workload("c2", scale=12, m=1 << 15, nbatch=2, batch=1000)
    h = hashlib.sha256()
    for a in (wl.graph.row_ptr, wl.graph.col, wl.graph.w):
        h.update(np.ascontiguousarray(a).tobytes())
    for b in wl.batches:
        h.update(b.records().tobytes())
    digest = torch.tensor(list(h.digest()[:8]), dtype=torch.int64)
    gathered = [torch.zeros_like(digest) for _ in range(world)]
    dist.all_gather(gathered, digest)
    same = all(torch.equal(gathered[0], x) for x in gathered)
    mx = bench.max_over_ranks(float(rank + 1))
    sm = bench.sum_over_ranks(float(10 * (rank + 1)))
    seeds = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(seeds, torch.tensor([bench.replica_seed(0, rank) & 0x7FFFFFFFFFFFFFFF], dtype=torch.int64))
    distinct = len({int(x.item()) for x in seeds}) == world
    out.put((rank, same, mx, sm, distinct))
    dist.destroy_process_group()


def test_replicas_share_inputs_and_reduce_timings():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, same, mx, sm, distinct in res:
        assert same, "replicas built different graphs or batches"
        assert mx == 2.0 and sm == 30.0
        assert distinct
