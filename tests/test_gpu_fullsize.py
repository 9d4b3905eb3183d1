"""Parity at the full sizes of the two largest workloads, on sampled vertices.

A whole export of RMAT-26 + hubs (about 70 GB of state) does not fit the host next to the oracle, but
the batch semantics are per source vertex (Section 5.2): a source's edges and groups depend only on
its own initial row and its own records.  So the oracle holds only the sampled sources' rows, with
the edge ids they have in the whole graph, and replays only their records with the insertion ids
the whole batch gives them; bingo_export_vertices exports the same vertices from the device, and the
two must agree bit for bit (adjacency, |G_k|, kinds, member sets) with the layout invariants holding.

- RMAT-26 + 64 hubs of 10^6 extra out-edges, uniform 31-bit biases: all 64 hubs and 10^4 uniform
  vertices, after creation, after a 10^6-record batch and after a 10^7-record batch; then the
  one-step law at the largest hub (10^6 samples, binned) and 10^5 PPR walks whose every step is a
  live edge of an oracle holding the visited sources.
- RMAT-24 with fixed-point biases: the 64 highest-degree vertices and 10^4 uniform vertices after
  creation; the workload's mixed node2vec + PPR launch (4M walkers) with every step of a sample of
  walks a live edge; and node2vec's second-order law (Eq. node2vec) at a (previous, current) vertex
  pair planted in this graph by an update batch, with neighbours at all three distances.
"""
import gc

import numpy as np
import pytest

import oracle as O
import workloads as W
from tests.gpu_helpers import (assert_state_matches, assert_vertices_match, insertion_ids, sampled_oracle)
from tests.stats import binned, chisq_p, tv

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import torch

    assert torch.cuda.is_available(), "GPU test"
    import paper_2504_10233_gb300 as B

    B.load()
    return B


def _t(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _release(*objs):
    import torch

    for o in objs:
        if hasattr(o, "close"):
            o.close()
    gc.collect()
    torch.cuda.empty_cache()


def test_export_vertices_rows_equal_the_whole_export(B):
    wl = W.make_workload("c2", scale=12, m=1 << 16, nbatch=1, batch=4000)
    G = wl.graph
    g = B.Graph(G.n, _t(G.row_ptr), _t(G.col), _t(G.w), max_bits=G.max_bits)
    g.apply_updates(_t(wl.batches[0].records()))
    ex = g.export_state()
    ids = np.concatenate([np.random.default_rng(3).permutation(G.n), [5, 5, G.n - 1]]).astype(np.uint32)
    exv = g.export_vertices(ids)
    for key in ("deg", "cnt", "kind", "one_slot", "glen", "sp_len"):
        assert (exv[key] == ex[key][ids]).all(), key
    eoff = np.concatenate([[0], np.cumsum(ex["deg"].astype(np.int64))])
    rows = np.concatenate([np.arange(eoff[v], eoff[v + 1]) for v in ids])
    for key in ("dst", "bias", "eid"):
        assert (exv[key] == ex[key][rows]).all(), key
    og = O.Graph(G.n, G.row_ptr, G.col, G.w)
    og.apply(wl.batches[0].records(), G.max_bits)
    assert_state_matches(ex, og)
    assert_vertices_match(exv, og, ids)
    with pytest.raises(B.BingoError):
        g.export_vertices(np.array([G.n], dtype=np.uint32))
    g.close()


def _sampled_parity_with_batches(B, wl, S, batch_sizes, seed=0):
    """Create, then apply the workload's records as consecutive batches of the given sizes; after
    creation and after every batch, the listed vertices must equal the sampled oracle's."""
    G = wl.graph
    rec = wl.batches[0].records()
    assert len(rec) >= sum(batch_sizes)
    g = B.Graph(G.n, _t(G.row_ptr), _t(G.col), _t(G.w), max_bits=G.max_bits)
    _release()
    og = sampled_oracle(G, S)
    assert_vertices_match(g.export_vertices(S), og, S)
    nxt = G.m
    off = 0
    for bs in batch_sizes:
        r = rec[off:off + bs]
        off += bs
        ids, nxt = insertion_ids(r, nxt)
        st = g.apply_updates(_t(r))
        sel = np.isin(r[:, 0], S)
        rc, ost = og.apply_ids(r[sel], ids[sel], G.max_bits)
        assert rc == 0
        assert st["inserted"] == int(((r[:, 3] == 0) | (r[:, 3] == 2)).sum())
        assert_vertices_match(g.export_vertices(S), og, S)
    g.check()
    return g, og, off


def test_c5_shape_sampled_parity_small(B):
    """The RMAT-26 + hubs recipe at scale 14 (hubs of 2^14 extra edges), the same machinery as the
    full-size test below: sampled vertices against the sampled oracle, whole state against the
    whole oracle."""
    wl = W.make_workload("c5", scale=14, m=1 << 18, nbatch=1, batch=30000)
    G = wl.graph
    hubs = np.asarray(wl.extra["hubs"], dtype=np.uint32)
    S = np.unique(np.concatenate([hubs, np.random.default_rng(1).integers(0, G.n, 500).astype(np.uint32)]))
    g, og, used = _sampled_parity_with_batches(B, wl, S, [3000, 27000])
    full = O.Graph(G.n, G.row_ptr, G.col, G.w)
    full.apply(wl.batches[0].records()[:3000], G.max_bits)
    full.apply(wl.batches[0].records()[3000:30000], G.max_bits)
    assert_state_matches(g.export_state(), full)
    g.close()


def test_c5_full_size_sampled_parity_law_and_live_steps(B):
    """RMAT-26 (2^26 vertices, 2^30 edges) + 64 hubs x 10^6, biases U[1, 2^31), at full size."""
    import torch

    wl = W.make_workload("c5", nbatch=1, batch=11_000_000)
    G = wl.graph
    assert G.n == 1 << 26 and G.m >= (1 << 30) + 64 * 10 ** 6 - 10 ** 7
    hubs = np.asarray(wl.extra["hubs"], dtype=np.uint32)
    assert len(hubs) == 64
    S = np.unique(np.concatenate([hubs, np.random.default_rng(26).integers(0, G.n, 10 ** 4).astype(np.uint32)]))
    g, og, used = _sampled_parity_with_batches(B, wl, S, [10 ** 6, 10 ** 7])
    rec = wl.batches[0].records()[:used]

    # one-step law at the largest hub after both batches
    offs, dst, w, _ = og.edges_of(hubs)
    hdeg = np.diff(offs.astype(np.int64))
    h = int(hubs[np.argmax(hdeg)])
    assert hdeg.max() > 9 * 10 ** 5
    a, b = int(offs[np.argmax(hdeg)]), int(offs[np.argmax(hdeg) + 1])
    cats, inv = np.unique(dst[a:b], return_inverse=True)
    probs = np.bincount(inv, weights=w[a:b].astype(np.float64), minlength=len(cats))
    N = 10 ** 6
    starts = torch.full((N,), h, dtype=torch.int32, device="cuda")
    paths = torch.empty((N, 2), dtype=torch.int32, device="cuda")
    plen = torch.empty(N, dtype=torch.int32, device="cuda")
    g.walk(starts, [B.policy(B.DEEPWALK, 1)], 99, 2, paths, plen)
    g.check()
    assert (plen.cpu().numpy() == 2).all()
    x = paths[:, 1].cpu().numpy().view(np.uint32)
    pos = np.searchsorted(cats, x)
    assert (cats[np.minimum(pos, len(cats) - 1)] == x).all(), "a step to a vertex that is not a neighbour"
    counts = np.bincount(pos, minlength=len(cats))
    assert tv(*binned(counts, probs, 256)) < 0.01
    assert chisq_p(*binned(counts, probs, 1000)) > 1e-3
    del starts, paths, plen

    # 10^5 PPR walks (stop 0.15, cap 100): every step a live edge after both batches
    nw = 10 ** 5
    st = _t(W.walk_starts(G.n, nw, 7))
    paths = torch.empty((nw, 101), dtype=torch.int32, device="cuda")
    plen = torch.empty(nw, dtype=torch.int32, device="cuda")
    g.walk(st, [B.policy(B.PPR, 100, 0.15)], 5, 101, paths, plen)
    g.check()
    P = paths.cpu().numpy().view(np.uint32)
    Lp = plen.cpu().numpy().astype(np.int64)
    g.close()
    del st, paths, plen
    _release()
    valid = np.arange(100)[None, :] < (Lp[:, None] - 1)
    u, xv = P[:, :-1][valid], P[:, 1:][valid]
    assert len(u) > 10 ** 5
    U = np.unique(u)
    ou = sampled_oracle(G, U)
    nxt = G.m
    for r in (rec[:10 ** 6], rec[10 ** 6:]):
        ids, nxt = insertion_ids(r, nxt)
        sel = np.isin(r[:, 0], U)
        assert ou.apply_ids(r[sel], ids[sel], G.max_bits)[0] == 0
    live = ou.count_edges(u, xv)
    assert (live > 0).all(), f"{int((live == 0).sum())} PPR steps are not live edges"


def _n2v_gadget(G, rng):
    """Records that plant, in the graph, a (previous a, current u) pair for node2vec's second-order
    law: a (3..8 edges of its own) gets four heavy edges to u (50..300 edges of its own), and u gets
    edges back to a (distance 0) and to every other neighbour of a (distance 1), next to its own,
    mostly distance-2, neighbours."""
    rp = G.row_ptr.astype(np.int64)
    deg = np.diff(rp)
    while True:
        a = int(rng.choice(np.nonzero((deg >= 3) & (deg <= 8))[0]))
        u = int(rng.choice(np.nonzero((deg >= 50) & (deg <= 300))[0]))
        na = set(int(x) for x in G.col[rp[a]:rp[a + 1]])
        if u != a and u not in na and a not in na:
            break
    rec = [(a, u, 25599, 0)] * 4 + [(u, a, 12800, 0)] * 2 + [(u, y, 20000, 0) for y in sorted(na)]
    return a, u, np.array(rec, dtype=np.uint32)


def test_c3_full_size_sampled_parity_mixed_launch_and_node2vec_law(B):
    """RMAT-24 (2^24 vertices, 2^28 edges), fixed-point biases in [128, 25600), at full size."""
    import torch

    wl = W.make_workload("c3")
    G = wl.graph
    assert G.n == 1 << 24 and G.m == 1 << 28
    deg = np.diff(G.row_ptr.astype(np.int64))
    top = np.argsort(-deg, kind="stable")[:64].astype(np.uint32)
    S = np.unique(np.concatenate([top, np.random.default_rng(24).integers(0, G.n, 10 ** 4).astype(np.uint32)]))
    g = B.Graph(G.n, _t(G.row_ptr), _t(G.col), _t(G.w), max_bits=G.max_bits)
    _release()
    assert_vertices_match(g.export_vertices(S), sampled_oracle(G, S), S)

    # the workload's launch: 4M walkers, node2vec (p=2, q=0.5, L=80) and PPR (0.15, cap 100) interleaved
    nw = wl.nwalkers
    pols = [B.policy(B.NODE2VEC, 80, n2v_pq=(2.0, 0.5)), B.policy(B.PPR, 100, 0.15)]
    starts = _t(W.walk_starts(G.n, nw, wl.walk_seed))
    pids = _t((np.arange(nw) % 2).astype(np.uint8))
    paths = torch.empty((nw, 101), dtype=torch.int32, device="cuda")
    plen = torch.empty(nw, dtype=torch.int32, device="cuda")
    g.walk(starts, pols, 3, 101, paths, plen, policy_ids=pids)
    g.check()
    Lp = plen.cpu().numpy().astype(np.int64)
    assert (Lp[0::2] <= 81).all() and (Lp[1::2] <= 101).all()
    samp = np.random.default_rng(5).choice(nw, size=20000, replace=False)
    P = paths[torch.from_numpy(samp).cuda()].cpu().numpy().view(np.uint32)
    Ls = Lp[samp]
    del starts, pids, paths, plen
    _release()
    valid = np.arange(100)[None, :] < (Ls[:, None] - 1)
    u, xv = P[:, :-1][valid], P[:, 1:][valid]
    assert (P[:, 0] == W.walk_starts(G.n, nw, wl.walk_seed)[samp]).all()
    # no updates in this workload: the live edges are the CSR rows
    U = np.unique(u).astype(np.int64)
    rp = G.row_ptr.astype(np.int64)
    d = rp[U + 1] - rp[U]
    rows = np.repeat(rp[U], d) + (np.arange(int(d.sum())) - np.repeat(np.cumsum(d) - d, d))
    keys = np.unique((np.repeat(U.astype(np.uint64), d) << np.uint64(32)) | G.col[rows].astype(np.uint64))
    q = (u.astype(np.uint64) << np.uint64(32)) | xv.astype(np.uint64)
    pos = np.minimum(np.searchsorted(keys, q), len(keys) - 1)
    assert (keys[pos] == q).all(), "a step that is not an edge"

    # node2vec's second-order law at a pair (a, u) planted by an update batch: the batch also updates
    # the edge index that the distance probes read (built by the launch above)
    a, u, rec = _n2v_gadget(G, np.random.default_rng(11))
    g.apply_updates(_t(rec))
    og = sampled_oracle(G, [a, u])
    ids, _ = insertion_ids(rec, G.m)
    assert og.apply_ids(rec, ids, G.max_bits)[0] == 0
    accept = [int(x) for x in pols[0].n2v_accept]
    offs, dst, wa, _ = og.edges_of([a])
    pu = float(wa[dst == u].sum()) / float(wa.sum())
    offs, dst, _, _ = og.edges_of([u])
    wts = og.n2v_weights(a, u, accept).astype(np.float64)
    cats, inv = np.unique(dst, return_inverse=True)
    probs = np.bincount(inv, weights=wts, minlength=len(cats))
    dist = np.array([0 if x == a else (1 if og.has_edge(a, int(x)) else 2) for x in cats])
    assert {0, 1, 2} <= set(dist.tolist()), "the pair must have neighbours at every distance"
    N = int(min(1 << 24, np.ceil(2.5e6 / pu)))
    starts = torch.full((N,), a, dtype=torch.int32, device="cuda")
    paths = torch.empty((N, 3), dtype=torch.int32, device="cuda")
    plen = torch.empty(N, dtype=torch.int32, device="cuda")
    g.walk(starts, [B.policy(B.NODE2VEC, 2, n2v_pq=(2.0, 0.5))], 17, 3, paths, plen)
    g.check()
    Pn = paths.cpu().numpy().view(np.uint32)
    sel = (Pn[:, 1] == u) & (plen.cpu().numpy() == 3)
    x2 = Pn[sel, 2]
    assert len(x2) >= 10 ** 6
    pos = np.searchsorted(cats, x2)
    assert (cats[np.minimum(pos, len(cats) - 1)] == x2).all()
    counts = np.bincount(pos, minlength=len(cats))
    assert tv(counts, probs) < 0.01
    assert chisq_p(counts, probs) > 1e-3
    g.close()
