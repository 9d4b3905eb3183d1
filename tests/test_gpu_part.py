"""1-D partitioned graphs and walks with walker migration (Supplement, partitioning).

The same walks on the whole graph and on its partitions: every path and length equal (walker w
draws from counters (w, step, j) wherever it runs), before and after an update batch routed to
the owners of its sources; walkers cross partitions (more than one superstep); each partition's
state equals the oracle's rows of its vertex range; plain walks on a partition graph are refused.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from tests.gpu_helpers import assert_vertices_match

pytestmark = pytest.mark.gpu


def _t(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module")
def B():
    import torch

    assert torch.cuda.is_available(), "GPU test"
    import paper_2504_10233_gb300 as B

    B.load()
    return B


def _walk(torch, g, starts, pols, pids, seed, stride):
    nw = len(starts)
    p = torch.full((nw, stride), -9, dtype=torch.int32, device="cuda")
    l = torch.zeros(nw, dtype=torch.int32, device="cuda")
    g.walk(starts, pols, seed, stride, p, l, policy_ids=pids)
    g.check()
    return p.cpu().numpy().view(np.uint32), l.cpu().numpy().view(np.uint32)


def _partition_oracle(G, lo, hi):
    """Oracle rows of [lo, hi) numbered as the partition numbers them: its own CSR order from 0."""
    rp = G.row_ptr.astype(np.int64)
    sub = np.zeros(G.n + 1, dtype=np.int64)
    sub[lo + 1:hi + 1] = np.diff(rp[lo:hi + 1])
    sub = np.cumsum(sub).astype(np.uint64)
    rows = np.arange(rp[lo], rp[hi])
    return O.Graph.from_csr_ids(G.n, sub, G.col[rows], G.w[rows], (rows - rp[lo]).astype(np.uint64), len(rows))


@pytest.mark.parametrize("nparts,explicit", [(2, False), (3, True)])
def test_partitioned_walks_equal_whole_graph_walks(B, nparts, explicit):
    import torch

    wl = W.make_workload("c2", scale=14, m=1 << 18, nbatch=1, batch=4000)
    G = wl.graph
    whole = B.Graph(G.n, _t(G.row_ptr), _t(G.col), _t(G.w), max_bits=G.max_bits, vertex_order=B.ORDER_CALLER)
    bounds = None
    if explicit:
        bounds = np.array([0, 1000, 9000, G.n], dtype=np.uint32)
    ps = B.PartitionedGraph(G.n, _t(G.row_ptr), _t(G.col), _t(G.w), nparts, bounds=bounds, max_bits=G.max_bits)
    nw, L = 20000, 40
    starts = _t(W.walk_starts(G.n, nw, 8))
    pids = _t((np.arange(nw) % 3).astype(np.uint8))
    pols = [B.policy(B.DEEPWALK, L), B.policy(B.PPR, L, 0.15), B.policy(B.NODE2VEC, L, n2v_pq=(2.0, 0.5))]
    rec = wl.batches[0].records()
    for phase in range(2):
        if phase == 1:
            st_w = whole.apply_updates(_t(rec))
            st_p = ps.apply_updates(_t(rec))
            for k in ("inserted", "deleted", "not_found"):
                assert st_w[k] == st_p[k], k
        for seed in (3, 4):
            pw, lw = _walk(torch, whole, starts, pols, pids, seed, L + 1)
            pp, lp = _walk(torch, ps, starts, pols, pids, seed, L + 1)
            assert (lw == lp).all(), "path lengths differ"
            assert (pw == pp).all(), "paths differ"
            assert ps.supersteps() > 2, "walkers must cross partitions"
    # each partition's state: the oracle's rows of its range, numbered as the partition numbers them
    for p in range(nparts):
        _, lo, hi = ps.part(p)
        og = _partition_oracle(G, lo, hi)
        mine = (rec[:, 0] >= lo) & (rec[:, 0] < hi)
        assert og.apply(rec[mine], G.max_bits)[0] == 0
        assert_vertices_match(ps.export_vertices(p, np.arange(hi - lo, dtype=np.uint32)), og,
                              np.arange(lo, hi, dtype=np.uint32))
    # plain walks on a partition graph are refused
    h, lo, hi = ps.part(0)
    st1 = _t(np.zeros(4, np.uint32))
    pth = torch.zeros((4, 3), dtype=torch.int32, device="cuda")
    ln = torch.zeros(4, dtype=torch.int32, device="cuda")
    with pytest.raises(B.BingoError) as e:
        B.bingo_walk(h, 4, st1, [pols[0]], 1, 3, pth, ln)
    assert e.value.status == B.E_STATE
    ps.close()
    whole.close()


def test_partition_arguments(B):
    wl = W.make_workload("c1")
    G = wl.graph
    for bounds in ([0, 0, G.n], [0, 600, 500, G.n], [1, 500, G.n]):
        with pytest.raises(B.BingoError):
            B.PartitionedGraph(G.n, G.row_ptr, G.col, G.w, len(bounds) - 1, bounds=bounds, max_bits=G.max_bits)
    ps = B.PartitionedGraph(G.n, G.row_ptr, G.col, G.w, 4, max_bits=G.max_bits)
    with pytest.raises(B.BingoError):  # a record with a source >= n rejects the whole batch
        ps.apply_updates(np.array([[0, 1, 3, 0], [G.n, 1, 3, 0]], dtype=np.uint32))
    ps.close()
