"""Internal vertex numbering: the graph's degree order against the caller's order.

The degree numbering only moves vertex records; every call takes and returns the
caller's ids and each vertex keeps its adjacency in the caller's CSR order.  So
both numberings must match the oracle after every batch, and the exported state
(layout included) and walks (bit-exact, every policy and launch form) must be the
same under both on a new graph and after insertions and streaming updates.  A
batch with deletions applies a vertex's deletions in internal-id order, so only
the canonical state is compared after one.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from tests.gpu_helpers import assert_state_matches, assert_steps_live
from tests.test_gpu_state import _stress_batch, _stress_graph

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import torch

    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2504_10233_gb300 import _build

    _build.build()
    import paper_2504_10233_gb300 as B

    B.load()
    return B


def dev(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def run_walk(B, g, starts, policies, seed, stride, pids=None, mode=0):
    import torch

    n = len(starts)
    paths = torch.empty((n, stride), dtype=torch.int32, device="cuda")
    plen = torch.empty(n, dtype=torch.int32, device="cuda")
    g.walk(dev(starts), policies, seed, stride, paths, plen, policy_ids=None if pids is None else dev(pids), mode=mode)
    g.check()
    return paths.cpu().numpy().view(np.uint32), plen.cpu().numpy().view(np.uint32)


def same_state(a, b):
    assert a.keys() == b.keys()
    for k in a:
        assert np.array_equal(np.asarray(a[k]), np.asarray(b[k])), k


def pols(B):
    return [B.policy(B.DEEPWALK, 20), B.policy(B.PPR, 30, 0.15), B.policy(B.NODE2VEC, 25, n2v_pq=(2.0, 0.5))]


def test_config_reports_the_numbering(B):
    og = _stress_graph(4)
    offs, dst, w, _ = og.edges()
    args = (og.n, dev(offs.astype(np.uint64)), dev(dst), dev(w))
    assert B.Graph(*args, max_bits=12).config().vertex_order == B.ORDER_DEGREE  # auto
    assert B.Graph(*args, max_bits=12, vertex_order=B.ORDER_CALLER).config().vertex_order == B.ORDER_CALLER
    assert B.Graph(*args, max_bits=12, vertex_order=B.ORDER_DEGREE).config().vertex_order == B.ORDER_DEGREE
    with pytest.raises(B.BingoError):
        B.Graph(*args, max_bits=12, vertex_order=3)


@pytest.mark.parametrize("stream", [False, True])
def test_state_and_updates_same_under_both_numberings(B, stream):
    og = _stress_graph(11)
    offs, dst, w, _ = og.edges()
    n = og.n
    gs = [B.Graph(n, dev(offs.astype(np.uint64)), dev(dst), dev(w), max_bits=12, vertex_order=o)
          for o in (B.ORDER_CALLER, B.ORDER_DEGREE)]
    same_state(gs[0].export_state(), gs[1].export_state())
    rng = np.random.default_rng(12)
    for it in range(8):
        rec = _stress_batch(rng, og, n, [5, 60, 300][it % 3])
        sts = [g.stream_updates(dev(rec)) if stream else g.apply_updates(dev(rec)) for g in gs]
        for r in ([x[None, :] for x in rec] if stream else [rec]):
            assert og.apply(r, 12)[0] == 0
        assert {k: sts[0][k] for k in ("inserted", "deleted", "not_found")} == \
               {k: sts[1][k] for k in ("inserted", "deleted", "not_found")}
        ex = [g.export_state() for g in gs]
        assert_state_matches(ex[0], og)
        assert_state_matches(ex[1], og)
        if stream:  # one record per step: the layout cannot depend on the numbering
            same_state(ex[0], ex[1])


def test_walks_identical_under_both_numberings(B):
    wl = W.make_workload("c2", scale=14, m=1 << 18, nbatch=2, batch=4000)
    G = wl.graph
    gs = [B.Graph(G.n, dev(G.row_ptr), dev(G.col), dev(G.w), max_bits=G.max_bits, vertex_order=o)
          for o in (B.ORDER_CALLER, B.ORDER_DEGREE)]
    nw = 20000
    starts = W.walk_starts(G.n, nw, 3)
    pids = (np.arange(nw) % 3).astype(np.uint8)
    og = O.Graph(G.n, G.row_ptr, G.col, G.w)
    ins = [b.records() for b in wl.batches]
    ins = [r[r[:, 3] == B.OP_INSERT] for r in ins]  # insertions keep the layouts equal
    for rec in ins:
        for mode in (0, B.WALK_STEPWISE):
            for lanes in (1, 4, 32):
                res = []
                for g in gs:
                    g.set_walk_config(lanes, 8, 0, 0)
                    res.append(run_walk(B, g, starts, pols(B), 77, 31, pids=pids, mode=mode))
                assert (res[0][0] == res[1][0]).all() and (res[0][1] == res[1][1]).all(), (mode, lanes)
        assert_steps_live(og, res[1][0], res[1][1])
        for g in gs:
            g.apply_updates(dev(rec))
        og.apply(rec, G.max_bits)
    # a batch with deletions: both graphs match the oracle and walk only live edges
    rec = wl.batches[0].records()
    rec = rec[rec[:, 3] != B.OP_INSERT]
    assert len(rec)
    for g in gs:
        g.apply_updates(dev(rec))
    og.apply(rec, G.max_bits)
    for g in gs:
        assert_state_matches(g.export_state(), og)
        paths, plen = run_walk(B, g, starts, pols(B), 78, 31, pids=pids)
        assert_steps_live(og, paths, plen)


def test_real_biases_same_under_both_numberings(B):
    rng = np.random.default_rng(5)
    n = 300
    edges = []
    for v in range(n):
        for _ in range(int(rng.integers(0, 40 if v % 17 else 400))):
            edges.append((v, int(rng.integers(0, n)), float(rng.choice([0.25, 1.5, 3.75, 100.125]))))
    og = O.Graph.from_edges(n, [(s, d, int(np.float32(x).view(np.uint32))) for s, d, x in edges])
    offs, dst, w, _ = og.edges()
    gs = [B.Graph(n, dev(offs.astype(np.uint64)), dev(dst), dev(w), bias_format=B.BIAS_F32, lambda_=2.0,
                  vertex_order=o) for o in (B.ORDER_CALLER, B.ORDER_DEGREE)]
    same_state(gs[0].export_state(), gs[1].export_state())
    assert np.array_equal(gs[0].export_decimal(), gs[1].export_decimal())
    starts = W.walk_starts(n, 50000, 8)
    res = [run_walk(B, g, starts, [B.policy(B.DEEPWALK, 15)], 3, 16) for g in gs]
    assert (res[0][0] == res[1][0]).all() and (res[0][1] == res[1][1]).all()
