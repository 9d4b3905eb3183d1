"""The seeded input generators produce the inputs the workload recipe states (no GPU).

The generators hold none of the method's arithmetic; these checks pin the properties the parity
tests and the bench rely on: ranges and laws of the biases, graph structure, the walk-start formula,
and the update protocol (the paper's hold-out protocol: insertions come from held-out edges,
deletions hit live edges, exact insert/delete counts per batch).
"""
import math

import numpy as np

import oracle as O
import workloads as W


def test_walk_starts_formula():
    n, seed = 1000, 7
    got = W.walk_starts(n, 64, seed)
    for i in range(64):
        x = int(W.philox4x32_10([i, 0, 0, 0], [seed & 0xFFFFFFFF, seed >> 32])[0])
        assert got[i] == (x * n) >> 32
    assert got.max() < n


def test_er_edges_in_range_without_self_loops():
    s, d = W.er_edges(1024, 50000, 3)
    assert len(s) == len(d) == 50000
    assert s.max() < 1024 and d.max() < 1024
    assert (s != d).all()
    deg = np.bincount(s, minlength=1024)
    assert deg.min() > 0 and deg.max() < 3 * deg.mean()  # uniform endpoints: no heavy tail


def test_rmat_edges_are_skewed_and_relabelled():
    s, d = W.rmat_edges(14, 1 << 18, 5)
    assert s.max() < 1 << 14 and d.max() < 1 << 14
    deg = np.bincount(s, minlength=1 << 14)
    assert deg.max() > 50 * deg.mean()  # power-law degrees
    assert (deg == 0).sum() > (1 << 14) // 10  # and many vertices without out-edges
    assert int(np.argmax(deg)) != 0  # the seeded relabelling moved RMAT's densest vertex off id 0


def test_pareto_biases_follow_the_floor_law():
    m, cap = 1_000_000, 1 << 20
    w = W.biases(m, ("pareto15", cap), 11).astype(np.int64)
    assert w.min() >= 1 and w.max() <= cap
    for k in (2, 4, 16, 64):
        p = k ** -1.5  # P(floor(U^(-1/1.5)) >= k) = P(U <= k^-1.5)
        got = float((w >= k).mean())
        assert abs(got - p) < 5 * math.sqrt(p * (1 - p) / m), (k, got, p)


def test_fixed_and_uniform_biases_ranges():
    f = W.biases(200_000, ("fixed", 128, 25600), 3).astype(np.int64)
    assert f.min() >= 128 and f.max() < 25600
    assert abs(f.mean() - (128 + 25599) / 2) < 0.01 * 25600
    u = W.biases(200_000, ("uniform", 1, 1 << 16), 4).astype(np.int64)
    assert u.min() >= 1 and u.max() < 1 << 16
    assert abs(u.mean() - (1 << 16) / 2) < 0.01 * (1 << 16)
    u31 = W.biases(200_000, ("uniform", 1, 1 << 31), 4).astype(np.int64)
    assert u31.min() >= 1 and u31.max() < 1 << 31 and u31.max() >= 1 << 30


def test_hub_edges():
    ids, s, d = W.hub_edges(1 << 12, 8, 500, 9)
    assert len(np.unique(ids)) == 8 and ids.max() < 1 << 12
    assert len(s) == 8 * 500 and set(np.unique(s).tolist()) == set(ids.tolist())
    assert (np.bincount(s, minlength=1 << 12)[ids] == 500).all()
    assert d.max() < 1 << 12


def test_c5_hub_edges_and_the_no_hub_option():
    """c5 at a small scale: the 64 hubs add their out-edges (capped at m/16 each at reduced scales) on
    top of the m RMAT edges; hubs=False (a profiling case) leaves them out and nothing else changes."""
    kw = dict(scale=12, m=1 << 16, nbatch=1, batch=2000)
    with_h = W.make_workload("c5", **kw)
    without = W.make_workload("c5", hubs=False, **kw)
    deg_h = np.diff(with_h.graph.row_ptr.astype(np.int64))
    deg_n = np.diff(without.graph.row_ptr.astype(np.int64))
    hubs = with_h.extra["hubs"]
    assert without.extra["hubs"] is None and len(hubs) == 64
    assert without.graph.m == 1 << 16 and with_h.graph.m == (1 << 16) + 64 * ((1 << 16) // 16)
    # the hold-out protocol keeps some hub edges back as insertions, so a hub's initial degree is a
    # little below its 4,096 generated edges, yet far above any vertex of the plain RMAT part
    assert deg_h[hubs].min() > deg_n.max() and deg_h[hubs].sum() > 0.9 * 64 * ((1 << 16) // 16)
    rec = without.batches[0].records()
    assert (rec[:, 3] == 0).sum() == 1000 and (rec[:, 3] == 1).sum() == 1000


def test_hold_out_protocol_batches():
    """c2's stream protocol: the created graph has exactly m edges, each batch holds the stated
    insert/delete counts, insertions are edges held out of the generated set, and every deletion
    finds a live edge when the batches are applied in order."""
    wl = W.make_workload("c2", scale=12, m=1 << 15, nbatch=3, batch=2000)
    G = wl.graph
    assert G.m == 1 << 15
    og = O.Graph(G.n, G.row_ptr, G.col, G.w)
    for b in wl.batches:
        rec = b.records()
        assert (rec[:, 3] == 0).sum() == 1000 and (rec[:, 3] == 1).sum() == 1000
        ins = rec[rec[:, 3] == 0]
        assert ins[:, 0].max() < G.n and ins[:, 1].max() < G.n and ins[:, 2].min() >= 1
        rc, (inserted, deleted, not_found) = og.apply(rec, G.max_bits)
        assert rc == 0 and inserted == 1000 and deleted == 1000 and not_found == 0


def test_uniform_batches_of_c1():
    """c1: insertions are new uniform edges without self-loops and with new biases in [1, 255];
    deletions are uniform over live edges."""
    wl = W.make_workload("c1")
    G = wl.graph
    og = O.Graph(G.n, G.row_ptr, G.col, G.w)
    rec = wl.batches[0].records()
    ins = rec[rec[:, 3] == 0]
    assert len(ins) == 1024 and (rec[:, 3] == 1).sum() == 1024
    assert (ins[:, 0] != ins[:, 1]).all() and ins[:, 2].min() >= 1 and ins[:, 2].max() <= 255
    rc, (inserted, deleted, not_found) = og.apply(rec, G.max_bits)
    assert rc == 0 and inserted == 1024 and deleted == 1024 and not_found == 0
