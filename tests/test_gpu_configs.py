"""Parity on the shapes of the c3, c4 and c5 workloads, through the C ABI (c1 and c2 have their own).

Each test keeps its workload's structure and shrinks only the scale:
  c3  RMAT, fixed-point biases w_fx in [128, 25600) (K = 15); one persistent launch mixing node2vec
      (p = 2, q = 0.5, length 80) and PPR (stop 0.15, cap 100) by walker id;
  c4  RMAT, uniform 16-bit biases; the held-out update stream (70% insertions) applied as streaming
      single-edge updates (each record a batch of one, Section 4.2); DeepWalk length 40;
  c5  RMAT with 64 injected hubs, uniform 31-bit biases (K = 31); 50/50 batches; PPR walkers.
The factorisation state after creation and after every update step must equal the oracle's
bit-exactly.  Walks are checked by properties that hold at any size: every step is a live edge; at
every position before the cap where the walker has an out-edge, a PPR walker stops with probability
exactly s (a binomial test over all such positions, since dead ends also end walks); node2vec walks
end early only at dead ends; and the persistent and step-by-step forms give identical paths.
"""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W
from tests.gpu_helpers import assert_state_matches, assert_steps_live
from tests.test_gpu_walk import B, dev, graph_of, one_step_check, run_walk  # noqa: F401  (B is a fixture)

pytestmark = pytest.mark.gpu


def oracle_of(G):
    return O.Graph(G.n, G.row_ptr, G.col, G.w)


def oracle_degrees(og):
    offs, _, _, _ = og.edges()
    return np.diff(offs.astype(np.int64))


def ppr_hazard_z(paths, plen, deg, cap, stop_u32):
    """z-score of the observed PPR stop rate against s = stop_u32 / 2^32.  A trial is a path
    position l < cap whose vertex has an out-edge (the stop test ran and, had it not stopped the
    walk, a step would follow); a success is a walk that ended at such a position."""
    s = stop_u32 / 2 ** 32
    steps = plen.astype(np.int64) - 1
    L = paths.shape[1]
    pos = np.arange(L)[None, :]
    on = pos <= steps[:, None]
    v = np.where(on, paths, 0).astype(np.int64)
    trials = int((on & (pos < cap) & (deg[v] > 0)).sum())
    last = paths[np.arange(len(paths)), steps].astype(np.int64)
    stops = int(((steps < cap) & (deg[last] > 0)).sum())
    assert trials > 10_000
    return (stops - trials * s) / math.sqrt(trials * s * (1 - s))


def test_c3_shape_state_and_mixed_launch(B):
    wl = W.make_workload("c3", scale=15, m=1 << 19)
    G = wl.graph
    assert G.max_bits == 15 and int(G.w.max()) < 25600 and int(G.w.min()) >= 128
    g = graph_of(B, G)
    og = oracle_of(G)
    assert_state_matches(g.export_state(), og)
    nw, stride = 1 << 16, 101
    starts = W.walk_starts(G.n, nw, wl.walk_seed)
    pids = (np.arange(nw) % 2).astype(np.uint8)  # node2vec and PPR interleaved by walker id
    pols = [B.policy(B.NODE2VEC, 80, n2v_pq=(2.0, 0.5)), B.policy(B.PPR, 100, 0.15)]
    paths, plen = run_walk(B, g, starts, pols, 0, stride, pids=pids)
    assert (paths[:, 0] == starts).all()
    assert_steps_live(og, paths, plen)
    deg = oracle_degrees(og)
    ppr = pids == 1
    z = ppr_hazard_z(paths[ppr], plen[ppr], deg, 100, pols[1].ppr_stop_u32)
    assert abs(z) < 4.5, z
    n2v = pids == 0
    st = plen[n2v].astype(np.int64) - 1
    early = st < 80
    last = paths[n2v][np.arange(int(n2v.sum())), st]
    assert (deg[last[early].astype(np.int64)] == 0).all(), "a node2vec walk ended early at a vertex with out-edges"
    step = run_walk(B, g, starts, pols, 0, stride, pids=pids, mode=B.WALK_STEPWISE)
    assert (step[0] == paths).all() and (step[1] == plen).all()


def test_c4_shape_streamed_update_stream(B):
    wl = W.make_workload("c4", scale=14, m=1 << 18, nbatch=2, batch=1500)
    G = wl.graph
    assert G.max_bits == 16
    g = graph_of(B, G)
    og = oracle_of(G)
    assert_state_matches(g.export_state(), og)
    nw, L = 1 << 14, wl.length
    starts = W.walk_starts(G.n, nw, wl.walk_seed)
    pol = [B.policy(B.DEEPWALK, L)]
    for ep, b in enumerate(wl.batches):
        rec = np.ascontiguousarray(b.records(), dtype=np.uint32)
        assert (rec[:, 3] == 0).sum() == round(0.7 * len(rec))  # 70% insertions
        st = g.stream_updates(dev(rec))
        tot = [0, 0, 0]
        for r in rec:  # the oracle applies the records one at a time, each a batch of one
            rc, s = og.apply(r[None, :], G.max_bits)
            assert rc == 0
            tot = [a + c for a, c in zip(tot, s)]
        assert (st["inserted"], st["deleted"], st["not_found"]) == tuple(tot), (st, tot)
        assert_state_matches(g.export_state(), og)
        paths, plen = run_walk(B, g, starts, pol, ep, L + 1)
        assert_steps_live(og, paths, plen)


def test_c5_shape_hubs_31bit_batches_and_ppr(B):
    wl = W.make_workload("c5", scale=14, m=1 << 18, nbatch=2, batch=4000)
    G = wl.graph
    assert G.max_bits == 31 and int(G.w.max()) >= 1 << 30
    hubs = np.asarray(wl.extra["hubs"], dtype=np.int64)
    assert len(hubs) == 64
    g = graph_of(B, G)
    og = oracle_of(G)
    assert_state_matches(g.export_state(), og)
    nw, cap = 1 << 16, 100
    starts = W.walk_starts(G.n, nw, wl.walk_seed)
    pol = B.policy(B.PPR, cap, 0.15)
    for ep, b in enumerate(wl.batches):
        rec = np.ascontiguousarray(b.records(), dtype=np.uint32)
        st = g.apply_updates(dev(rec))
        rc, ost = og.apply(rec, G.max_bits)
        assert rc == 0 and (st["inserted"], st["deleted"], st["not_found"]) == ost, (st, ost)
        assert_state_matches(g.export_state(), og)
        paths, plen = run_walk(B, g, starts, [pol], ep, cap + 1)
        assert_steps_live(og, paths, plen)
        z = ppr_hazard_z(paths, plen, oracle_degrees(og), cap, pol.ppr_stop_u32)
        assert abs(z) < 4.5, z
    deg = oracle_degrees(og)
    hub = int(hubs[np.argmax(deg[hubs])])
    assert deg[hub] > 16384
    one_step_check(B, g, og, hub, 5)  # 31-bit biases at a hub: nearly every group dense (rejection)
