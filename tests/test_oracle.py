"""Pins for the CPU oracle against what the paper and the mathematics fix.

Worked examples (tests/golden/*.json, each citing its passage), Theorem 1 in
exact rationals by brute force on tiny vertices, the ITS sampler by exhaustive
enumeration of r, closed forms (truncated geometric PPR lengths, node2vec on a
tiny graph), special cases and the invariant sum_k 2^k |G_k| = sum w.
"""
import itertools
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
import workloads as W
from tests.conftest import golden
from tests.stats import binned, chisq_p, tv

KIND = {"empty": O.EMPTY, "dense": O.DENSE, "one": O.ONE, "sparse": O.SPARSE, "regular": O.REGULAR}


def _groups_by_dst(g, v):
    """{k: sorted dst list} for vertex v through the oracle's membership export."""
    offs, dst, w, eid = g.edges()
    eid2dst = {int(e): int(d) for e, d in zip(eid, dst)}
    moffs, meids = g.members_all()
    out = {}
    for k in range(32):
        a, b = int(moffs[32 * v + k]), int(moffs[32 * v + k + 1])
        if b > a:
            out[k] = sorted(eid2dst[int(e)] for e in meids[a:b])
    return out


def test_running_example_groups_totals_insert_delete():
    gd = golden("running_example.json")
    n = 6
    g = O.Graph.from_edges(n, [tuple(e) for e in gd["edges"]])
    v = gd["vertex"]
    grp = _groups_by_dst(g, v)
    assert grp == {int(k): sorted(x) for k, x in gd["groups"].items()}
    Wk = g.group_totals(v)
    for k, t in gd["totals"].items():
        assert int(Wk[int(k)]) == t
    cnt, _, sw = g.factor(v)
    assert sum(int(cnt[k]) << k for k in range(32)) == sw == 12
    # insertion example
    s, d, b = gd["insert"]["edge"]
    rc, st = g.apply(np.array([[s, d, b, 0]]))
    assert rc == 0 and st == (1, 0, 0)
    assert _groups_by_dst(g, v) == {int(k): sorted(x) for k, x in gd["insert"]["groups_after"].items()}
    # deletion example: the deleted edge is neighbour index 0 and touches groups 2^0 and 2^2
    offs, dst, w, eid = g.edges()
    s, d, b = gd["delete"]["edge"]
    row = list(zip(dst[offs[v]:offs[v + 1]], w[offs[v]:offs[v + 1]]))
    assert row.index((d, b)) == gd["delete"]["neighbor_index"]
    assert [k for k in range(32) if b & (1 << k)] == gd["delete"]["groups_touched"]
    rc, st = g.apply(np.array([[s, d, 0, 1]]))
    assert rc == 0 and st == (0, 1, 0)
    assert _groups_by_dst(g, v) == {int(k): sorted(x) for k, x in gd["delete"]["groups_after"].items()}


def test_float_example():
    gd = golden("float_example.json")
    cnt, ndec, wi, wd = O.float_factor(gd["biases"], gd["lambda"])
    for k, members in gd["groups"].items():
        assert int(cnt[int(k)]) == len(members)
    assert ndec == len(gd["decimal_group"])
    assert abs(wd / (wi + wd) - gd["decimal_share"]) < 1e-12
    # membership: neighbour j is in group k iff bit k of floor(lambda * b_j) is set
    ip = [int(np.floor(gd["lambda"] * b)) for b in gd["biases"]]
    assert ip == [5, 7, 3]


def test_adaption_example():
    gd = golden("adaption_example.json")
    g = O.Graph.from_edges(1 + gd["d"], [(0, 1 + j, b) for j, b in enumerate(gd["biases"])])
    cnt, kd, sw = g.factor(0, gd["alpha"], gd["beta"])
    for k, c in gd["counts"].items():
        assert int(cnt[int(k)]) == c
    for k, name in gd["kinds"].items():
        assert int(kd[int(k)]) == KIND[name], k
    # the neighbour rejected for group 2^0 is not a member of it, and Theorem 1 still holds for it
    grp = _groups_by_dst(g, 0)
    for j in gd["rejected_for_group0"]:
        assert (1 + j) not in grp[0]
    for i, b in enumerate(gd["biases"]):
        assert Fraction(*g.factored_prob(0, i, gd["alpha"], gd["beta"])) == Fraction(b, sw)


def test_kind_boundaries():
    for case in golden("kind_boundaries.json")["cases"]:
        assert O.kind(case["cnt"], case["d"]) == KIND[case["kind"]], case


def test_update_semantics():
    gd = golden("update_semantics.json")
    g = O.Graph.from_edges(gd["n"], [tuple(e) for e in gd["initial"]])
    for b in gd["batches"]:
        rc, st = g.apply(np.array(b["records"], dtype=np.uint32), max_bits=32)
        if b.get("status") == "invalid":
            assert rc == 1, b["why"]
        else:
            assert rc == 0 and list(st) == b["stats"], b["why"]
        offs, dst, w, eid = g.edges()
        for v in range(gd["n"]):
            got = [[int(dst[j]), int(w[j]), int(eid[j])] for j in range(int(offs[v]), int(offs[v + 1]))]
            exp = b["edges_after"].get(str(v), [])
            assert got == exp, (b["why"], v)


def _batch_by_definition(lists, next_eid, rec):
    """Section 5.2's batch semantics written out: every insertion in batch order (new ids continue
    the count), then every deletion in batch order, each removing the live copy of (src, dst) with
    the smallest edge id; a bias change is one insertion plus one deletion."""
    for s_, d_, b_, op in rec:
        if op in (0, 2):
            lists[s_].append((d_, b_, next_eid))
            next_eid += 1
    nf = 0
    for s_, d_, b_, op in rec:
        if op in (1, 2):
            hit = [e for e in lists[s_] if e[0] == d_]
            if not hit:
                nf += 1
                continue
            lists[s_].remove(min(hit, key=lambda e: e[2]))
    return next_eid, nf


def test_batch_semantics_brute_force():
    """Random tiny multigraphs with many duplicate (src, dst) pairs and batches mixing all three
    operations: the oracle's adjacency equals the semantics written out in plain Python."""
    rng = np.random.default_rng(17)
    for trial in range(40):
        n = 5
        edges = [(int(rng.integers(0, n)), int(rng.integers(0, 3)), int(rng.integers(1, 16))) for _ in range(25)]
        g = O.Graph.from_edges(n, edges)
        lists = {v: [] for v in range(n)}
        for eid_, (_, (s_, d_, b_)) in enumerate(sorted(enumerate(edges), key=lambda t: (t[1][0], t[0]))):
            lists[s_].append((d_, b_, eid_))  # edge ids follow the CSR order
        nxt = len(edges)
        for _ in range(3):
            rec = [(int(rng.integers(0, n)), int(rng.integers(0, 3)), int(rng.integers(1, 16)), int(rng.integers(0, 3)))
                   for _ in range(int(rng.integers(1, 30)))]
            rc, st = g.apply(np.array(rec, dtype=np.uint32))
            nxt, nf = _batch_by_definition(lists, nxt, rec)
            assert rc == 0 and st[2] == nf
            offs, dst, w, eid = g.edges()
            for v in range(n):
                got = [(int(dst[j]), int(w[j]), int(eid[j])) for j in range(int(offs[v]), int(offs[v + 1]))]
                assert got == lists[v], (trial, v)


def test_sampled_sources_replay_equals_full_replay():
    """A graph holding only some sources' rows, with their edge ids, that replays only those sources'
    records with the insertion ids they have in the whole batch ends with the same edges as the whole
    graph (batch semantics are per source, Section 5.2)."""
    wl = W.make_workload("c1")
    G = wl.graph
    full = O.Graph(G.n, G.row_ptr, G.col, G.w)
    rp = G.row_ptr.astype(np.int64)
    eid_all = np.arange(rp[-1], dtype=np.uint64)
    same = O.Graph.from_csr_ids(G.n, G.row_ptr, G.col, G.w, eid_all, rp[-1])
    assert all((a == b).all() for a, b in zip(same.edges(), full.edges()))
    S = np.array([0, 3, 17, 200, 511, G.n - 1], dtype=np.uint32)
    deg = rp[S + 1] - rp[S]
    sub_rp = np.zeros(G.n + 1, dtype=np.uint64)
    sub_rp[S.astype(np.int64) + 1] = deg
    sub_rp = np.cumsum(sub_rp).astype(np.uint64)
    rows = np.concatenate([np.arange(rp[v], rp[v + 1]) for v in S])
    sub = O.Graph.from_csr_ids(G.n, sub_rp, G.col[rows], G.w[rows], rows.astype(np.uint64), rp[-1])
    rec = wl.batches[0].records()
    # duplicate deletions and bias changes of sampled sources too
    extra = np.array([[int(S[1]), int(G.col[rp[S[1]]]), 0, 1]] * 3 + [[int(S[2]), int(G.col[rp[S[2]]]), 9, 2]],
                     dtype=np.uint32)
    rec = np.concatenate([rec, extra])
    nxt = full.m
    ins = (rec[:, 3] == 0) | (rec[:, 3] == 2)
    ids = (nxt + np.cumsum(ins) - 1).astype(np.uint64)
    assert full.apply(rec)[0] == 0
    sel = np.isin(rec[:, 0], S)
    assert sub.apply_ids(rec[sel], ids[sel])[0] == 0
    a, b = full.edges_of(S), sub.edges_of(S)
    assert all((x == y).all() for x, y in zip(a, b))


def test_count_edges_equals_has_edge():
    """The batched live-copy count against the plain list scan (o_has_edge) and a count of the
    exported adjacency, on c1 after its batch."""
    wl = W.make_workload("c1")
    G = wl.graph
    g = O.Graph(G.n, G.row_ptr, G.col, G.w)
    g.apply(wl.batches[0].records(), G.max_bits)
    offs, dst, _, _ = g.edges()
    rng = np.random.default_rng(9)
    us = rng.integers(0, G.n, 20000).astype(np.uint32)
    xs = rng.integers(0, G.n, 20000).astype(np.uint32)
    live = np.repeat(np.arange(G.n), np.diff(offs.astype(np.int64)))
    us[:5000], xs[:5000] = live[:5000], dst[:5000]  # pairs that exist
    got = g.count_edges(us, xs)
    for u, x, c in zip(us[::7], xs[::7], got[::7]):
        seg = dst[int(offs[u]):int(offs[u + 1])]
        assert c == int((seg == x).sum()) and (c > 0) == g.has_edge(int(u), int(x))
    assert (got[:5000] > 0).all()


def test_philox_known_answers():
    for vec in golden("philox_kat.json")["vectors"]:
        out = W.philox4x32_10([int(x, 16) for x in vec["ctr"]], [int(x, 16) for x in vec["key"]])
        assert [int(x) for x in out] == [int(x, 16) for x in vec["out"]]


def test_node2vec_tiny_closed_form():
    gd = golden("node2vec_tiny.json")
    g = O.Graph.from_edges(gd["n"], [tuple(e) for e in gd["edges"]])
    ss = gd["second_step"]
    wts = g.n2v_weights(ss["prev"], ss["u"], gd["accept_u32"])
    offs, dst, _, _ = g.edges()
    nb = [int(x) for x in dst[offs[ss["u"]]:offs[ss["u"] + 1]]]
    assert nb == ss["neighbors"]
    tot = int(wts.sum())
    assert [Fraction(int(x), tot) for x in wts] == [Fraction(a, ss["prob_den"]) for a in ss["prob_num"]]
    # walk frequencies of 2-step node2vec paths from vertex 0
    tp = gd["two_step_paths_from_0"]
    pol = O.policy(O.NODE2VEC, 2, 0, gd["accept_u32"])
    N = 200_000
    paths, plen = g.walk(np.zeros(N, dtype=np.uint32), [pol], seed=11)
    assert (plen == 3).all()
    keys = [tuple(p) for p in tp["paths"]]
    idx = {k: i for i, k in enumerate(keys)}
    counts = np.zeros(len(keys))
    for row in paths:
        counts[idx[tuple(int(x) for x in row)]] += 1
    probs = np.array(tp["prob_num"], dtype=np.float64) / tp["prob_den"]
    assert tv(counts, probs) < 0.01
    assert chisq_p(counts, probs) > 1e-3


def _vertex_graph(configs):
    """One vertex per bias configuration; vertex v's edges go to arbitrary targets."""
    edges = []
    n = len(configs) + 8
    for v, ws in enumerate(configs):
        for j, w in enumerate(ws):
            edges.append((v, (v + j + 1) % n, w))
    return O.Graph.from_edges(n, edges)


def test_theorem1_exact_exhaustive_small():
    configs = [c for d in (1, 2, 3) for c in itertools.product(range(1, 16), repeat=d)]
    g = _vertex_graph(configs)
    for v, ws in enumerate(configs):
        s = sum(ws)
        for i, w in enumerate(ws):
            assert Fraction(*g.factored_prob(v, i)) == Fraction(w, s), (ws, i)


def test_theorem1_exact_random_up_to_d6():
    rng = np.random.default_rng(5)
    configs = [tuple(int(x) for x in rng.integers(1, 64, size=int(rng.integers(4, 7)))) for _ in range(1500)]
    # plus vertices whose groups cover all four kinds
    configs += [tuple([1] * 9 + [2, 6]), tuple([1] * 30 + [3, 3]), tuple([7] * 3 + [1] * 40 + [64, 128])]
    g = _vertex_graph(configs)
    kinds_seen = set()
    for v, ws in enumerate(configs):
        _, kd, _ = g.factor(v)
        kinds_seen |= set(int(x) for x in kd)
        s = sum(ws)
        for i, w in enumerate(ws):
            assert Fraction(*g.factored_prob(v, i)) == Fraction(w, s)
    assert {O.DENSE, O.ONE, O.SPARSE, O.REGULAR} <= kinds_seen


def test_its_exhaustive_enumeration():
    rng = np.random.default_rng(7)
    configs = [tuple(int(x) for x in rng.integers(1, 40, size=int(rng.integers(1, 7)))) for _ in range(120)]
    g = _vertex_graph(configs)
    for v, ws in enumerate(configs):
        hits = [0] * len(ws)
        for r in range(sum(ws)):
            hits[g.its_pick(v, r)] += 1
        assert hits == list(ws)


def test_special_cases_uniform_and_powers_of_two():
    # all biases 1: one group (k = 0) holding every edge -> uniform sampling
    g = O.Graph.from_edges(12, [(0, j + 1, 1) for j in range(10)])
    cnt, kd, sw = g.factor(0)
    assert int(cnt[0]) == 10 and int(cnt[1:].sum()) == 0 and kd[0] == O.DENSE
    assert all(Fraction(*g.factored_prob(0, i)) == Fraction(1, 10) for i in range(10))
    # distinct powers of two: every edge alone in its own group
    g = O.Graph.from_edges(12, [(0, j + 1, 1 << j) for j in range(10)])
    cnt, kd, sw = g.factor(0)
    assert [int(x) for x in cnt[:10]] == [1] * 10 and int(cnt[10:].sum()) == 0
    assert all(kd[k] == O.ONE for k in range(10))
    assert sw == (1 << 10) - 1


def test_invariants_after_random_batches():
    wl = W.make_workload("c1")
    G = wl.graph
    g = O.Graph(G.n, G.row_ptr, G.col, G.w)
    m0 = g.m
    for b in wl.batches:
        rc, (ins, dele, nf) = g.apply(b.records(), G.max_bits)
        assert rc == 0
        assert g.m == m0 + ins - dele
        m0 = g.m
    cnt, kd, sw = g.factor_all()
    offs, dst, w, eid = g.edges()
    deg = np.diff(offs.astype(np.int64))
    tot = (cnt.astype(np.uint64) << np.arange(32, dtype=np.uint64)[None, :]).sum(axis=1)
    assert (tot == sw).all()
    for v in range(0, G.n, 97):
        Wk = g.group_totals(v)
        assert all(int(Wk[k]) == int(cnt[v, k]) << k for k in range(32))
        assert all(int(kd[v, k]) == O.kind(int(cnt[v, k]), int(deg[v])) for k in range(32))
    assert len(np.unique(eid)) == len(eid)


def test_oracle_sampler_statistics():
    wl = W.make_workload("c1")
    G = wl.graph
    g = O.Graph(G.n, G.row_ptr, G.col, G.w)
    offs, dst, w, eid = g.edges()
    for v in (0, 17, 511):
        a, b = int(offs[v]), int(offs[v + 1])
        s = g.sample_many(v, 1_000_000, seed=v + 1)
        counts = np.bincount(s.astype(np.int64), minlength=b - a)
        probs = w[a:b].astype(np.float64)
        assert tv(counts, probs) < 0.01
        assert chisq_p(counts, probs) > 1e-3


def _one_step_counts(g, starts, seed, pol):
    """Destination of the first step of o_walk from every start (length-1 walks)."""
    paths, plen = g.walk(starts, [pol], seed=seed)
    assert (plen == 2).all(), "every start has out-edges, so every length-1 walk takes its step"
    return paths[:, 1]


def test_oracle_walk_first_order_law():
    """o_walk's first-order next hop (inverse transform over the walk's per-vertex u64 prefix
    sums, the path every DeepWalk and PPR step and node2vec's first step take) against the
    transition probability w_i / sum w of Section 2.1.  Several start vertices share one call,
    including the first and last vertex of the graph, so each reads its own slice of the walk's
    prefix-sum table.  Hubs with d > 1,000 are binned in edge order with exact bin masses (TV on
    256 bins, chi-square on 1,000), and a hub with 31-bit biases has a total above 2^32."""
    wl = W.make_workload("c1")
    G = wl.graph
    g = O.Graph(G.n, G.row_ptr, G.col, G.w)
    offs, dst, w, eid = g.edges()
    vs = [0, 17, 511, G.n - 1]
    N = 1_000_000
    starts = np.repeat(np.array(vs, dtype=np.uint32), N)
    for kind, n_pol in ((O.DEEPWALK, O.policy(O.DEEPWALK, 1)), (O.NODE2VEC, O.policy(O.NODE2VEC, 1, 0, (1 << 30, 1 << 31, 1 << 32)))):
        x = _one_step_counts(g, starts, 11 + kind, n_pol)
        for i, v in enumerate(vs):
            a, b = int(offs[v]), int(offs[v + 1])
            cats, inv = np.unique(dst[a:b], return_inverse=True)  # duplicates merged by summing weight
            probs = np.bincount(inv, weights=w[a:b].astype(np.float64), minlength=len(cats))
            xs = x[i * N:(i + 1) * N]
            assert np.isin(xs, cats).all()
            counts = np.bincount(np.searchsorted(cats, xs), minlength=len(cats))
            assert tv(counts, probs) < 0.01, (kind, v)
            assert chisq_p(counts, probs) > 1e-3, (kind, v)

    # hubs: distinct destinations, so a sampled destination names its edge
    rng = np.random.default_rng(5)
    d = 5000
    n = d + 3
    hub_w = [rng.integers(1, 1 << 20, size=d), rng.integers(1, 1 << 31, size=d)]
    edges = []
    for h, ws in enumerate(hub_w):
        edges += [(h, 3 + j, int(ws[j])) for j in range(d)]
    edges += [(2, 0, 1), (2, 1, 3)] + [(3 + j, 2, 1) for j in range(d)]
    g = O.Graph.from_edges(n, edges)
    assert sum(int(x) for x in hub_w[1]) > 1 << 32
    starts = np.repeat(np.array([0, 1], dtype=np.uint32), N)
    x = _one_step_counts(g, starts, 23, O.policy(O.DEEPWALK, 1))
    for h, ws in enumerate(hub_w):
        counts = np.bincount(x[h * N:(h + 1) * N].astype(np.int64) - 3, minlength=d)
        assert counts.sum() == N and len(counts) == d
        probs = ws.astype(np.float64)
        assert tv(*binned(counts, probs, 256)) < 0.01, h
        assert chisq_p(*binned(counts, probs, 1000)) > 1e-3, h


def test_ppr_length_truncated_geometric():
    # a ring with chords: every vertex has out-edges, so only the stop rule ends walks
    n = 64
    edges = [(v, (v + 1) % n, 1 + v % 5) for v in range(n)] + [(v, (v * 7 + 3) % n, 2) for v in range(n)]
    g = O.Graph.from_edges(n, edges)
    s_u32 = 644245094  # round(0.15 * 2^32)
    cap = 30
    pol = O.policy(O.PPR, cap, s_u32)
    N = 400_000
    starts = W.walk_starts(n, N, 3)
    _, plen = g.walk(starts, [pol], seed=5)
    steps = plen.astype(np.int64) - 1
    counts = np.bincount(steps, minlength=cap + 1)
    s = s_u32 / 2 ** 32
    probs = np.array([(1 - s) ** l * s for l in range(cap)] + [(1 - s) ** cap])
    assert abs(probs.sum() - 1) < 1e-12
    assert chisq_p(counts, probs) > 1e-3
    assert tv(counts, probs) < 0.01


def test_oracle_walk_steps_are_live_edges_and_padding():
    wl = W.make_workload("c1")
    G = wl.graph
    g = O.Graph(G.n, G.row_ptr, G.col, G.w)
    starts = W.walk_starts(G.n, 256, 0)
    paths, plen = g.walk(starts, [O.policy(O.DEEPWALK, 80)], seed=1)
    for i in range(256):
        L = int(plen[i])
        assert paths[i, 0] == starts[i]
        for t in range(L - 1):
            assert g.has_edge(int(paths[i, t]), int(paths[i, t + 1]))
        assert (paths[i, L:] == O.PAD).all()


# ----------------------------------------------------------------------------- real-valued biases


def _f32_bits(xs):
    return [int(b) for b in np.asarray(xs, dtype=np.float32).view(np.uint32)]


def _real_vertex_graph(configs, lam):
    """One source vertex per config (a tuple of binary32 biases), neighbours 0.. in order."""
    n = len(configs) + max(len(c) for c in configs)
    edges = [(v, len(configs) + j, b) for v, ws in enumerate(configs) for j, b in enumerate(_f32_bits(ws))]
    g = O.Graph.from_edges(n, edges)
    assert g.set_lambda(lam) == 0
    return g


def test_real_bias_worked_example():
    """Section 4.3 / Fig. SAMPLING2: lambda = 10 scales 0.554, 0.726, 0.320 to 5.54, 7.26, 3.20;
    integer parts 5, 7, 3 give groups 2^0 = {1,4,5}, 2^1 = {4,5}, 2^2 = {1,4}; every decimal part
    is nonzero, so the decimal group is {1,4,5}; W_D / (W_I + W_D) = 1/16."""
    gd = golden("float_example.json")
    g = O.Graph.from_edges(6, [(2, d, b) for d, b in zip(gd["neighbors"], _f32_bits(gd["biases"]))])
    assert g.set_lambda(gd["lambda"]) == 0
    I, q, qsum = g.real_parts()
    assert [int(x) for x in I] == gd["integer_parts"]
    assert _groups_by_dst(g, 2) == {int(k): sorted(x) for k, x in gd["groups"].items()}
    offs, dst, _, _ = g.edges()
    assert sorted(int(d) for d, qq in zip(dst, q) if qq > 0) == gd["decimal_group"]
    # decimal parts kept to 2^-8: within one unit of the printed scaled values' fractions
    for qq, x in zip(q, gd["scaled"]):
        assert abs(int(qq) / 256 - (x - int(x))) < 1 / 256
    WI, WD = sum(int(x) for x in I), int(qsum[2]) / 256
    assert abs(WD / (WI + WD) - gd["decimal_share"]) < 1e-3
    # group totals in units of 2^-8, decimal total in slot 31
    Wk = g.group_totals(2)
    assert [int(Wk[k]) for k in range(3)] == [256 * 3 * 1, 256 * 2 * 2, 256 * 2 * 4]
    assert int(Wk[31]) == int(qsum[2])


def test_real_bias_weight_is_floor_of_scaled_value():
    """When lambda * b is exact in binary64 (short mantissas, small integer lambda) the two parts
    recombine to floor(2^8 lambda b), computed here in exact rationals."""
    rng = np.random.default_rng(11)
    mant = rng.integers(1, 1 << 12, size=400)
    expo = rng.integers(-14, 10, size=400)
    bs = np.ldexp(mant.astype(np.float64), expo).astype(np.float32)
    bs = bs[(bs > 0) & (bs < 1e5)]
    for lam in (1.0, 3.0, 10.0, 1000.0):
        keep = [float(b) for b in bs if 256 * lam * float(b) >= 1 and lam * float(b) < 2**31]
        g = _real_vertex_graph([tuple(keep)], lam)
        I, q, _ = g.real_parts()
        for b, ii, qq in zip(keep, I, q):
            exact = Fraction(b) * Fraction(lam) * 256
            assert (int(ii) << 8) + int(qq) == exact.numerator // exact.denominator


def test_real_bias_theorem1_exact():
    """Integer groups weighted 2^8 2^k |G_k| plus the decimal group weighted Q_D with members drawn
    by q_i / Q_D give every neighbour probability (2^8 I_i + q_i) / sum (the decomposition loses
    nothing): exact rationals, including vertices whose biases are all below 1/lambda."""
    rng = np.random.default_rng(12)
    for lam in (1.0, 10.0, 37.5):
        configs = [tuple(rng.uniform(0.5, 100.0, size=int(rng.integers(1, 7))).astype(np.float32)) for _ in range(300)]
        configs += [tuple(rng.uniform(0.01, 0.99, size=int(rng.integers(1, 7))).astype(np.float32) / lam)
                    for _ in range(100)]
        configs = [c for c in configs if all(256 * lam * float(b) >= 1 for b in c)]
        g = _real_vertex_graph(configs, lam)
        I, q, _ = g.real_parts()
        offs, _, _, _ = g.edges()
        decimal_only = 0
        for v, ws in enumerate(configs):
            a, b = int(offs[v]), int(offs[v + 1])
            wts = [(int(I[j]) << 8) + int(q[j]) for j in range(a, b)]
            decimal_only += all(int(I[j]) == 0 for j in range(a, b))
            for i in range(b - a):
                assert Fraction(*g.factored_prob(v, i)) == Fraction(wts[i], sum(wts)), (lam, ws, i)
        assert decimal_only > 50


def test_real_bias_its_enumeration():
    rng = np.random.default_rng(13)
    configs = [tuple(rng.uniform(0.05, 3.0, size=int(rng.integers(1, 5))).astype(np.float32)) for _ in range(60)]
    g = _real_vertex_graph(configs, 2.0)
    I, q, _ = g.real_parts()
    offs, _, _, _ = g.edges()
    for v in range(len(configs)):
        a, b = int(offs[v]), int(offs[v + 1])
        wts = [(int(I[j]) << 8) + int(q[j]) for j in range(a, b)]
        hits = [0] * len(wts)
        for r in range(sum(wts)):
            hits[g.its_pick(v, r)] += 1
        assert hits == wts


def test_real_bias_validation():
    bad = [float("nan"), float("inf"), -1.0, 0.0, 1e-9, 3e9]
    for b in bad:
        g = O.Graph.from_edges(3, [(0, 1, _f32_bits([b])[0])])
        assert g.set_lambda(1.0) != 0, b
    g = O.Graph.from_edges(3, [(0, 1, _f32_bits([1.5])[0])])
    assert g.set_lambda(1.0) == 0
    for b in bad:
        rc, _ = g.apply(np.array([[0, 2, _f32_bits([b])[0], 0]], dtype=np.uint32))
        assert rc != 0, b
    rc, st = g.apply(np.array([[0, 2, _f32_bits([0.25])[0], 0]], dtype=np.uint32))
    assert rc == 0 and st == (1, 0, 0)
    I, q, qsum = g.real_parts()
    assert [int(x) for x in I] == [1, 0] and [int(x) for x in q] == [128, 64] and int(qsum[0]) == 192


def test_baseline_all_regular():
    """Section 6.2 (Fig. Moptimization): the BS baseline keeps every group in regular format.  The
    factorisation (counts, memberships) is unchanged, every nonempty group is regular, and the
    sampler still draws w / sum w (Theorem 1 does not depend on the representation)."""
    rng = np.random.default_rng(21)
    configs = [tuple(int(x) for x in rng.integers(1, 64, size=int(rng.integers(1, 9)))) for _ in range(400)]
    configs += [tuple([1] * 9 + [2, 6]), tuple([1] * 30 + [3, 3]), tuple([7] * 3 + [1] * 40 + [64, 128])]
    g = _vertex_graph(configs)
    for v, ws in enumerate(configs):
        cnt_ga, kd_ga, sw = g.factor(v)
        cnt, kd, sw2 = g.factor(v, O.ALL_REGULAR, 0)
        assert (cnt == cnt_ga).all() and sw == sw2 == sum(ws)
        assert all(int(kd[k]) == (O.REGULAR if cnt[k] else O.EMPTY) for k in range(32))
        for i, w in enumerate(ws):
            assert Fraction(*g.factored_prob(v, i, O.ALL_REGULAR, 0)) == Fraction(w, sum(ws))
    # the last vertex has dense and one-element groups under Eq. group (and none under BS, above)
    assert {int(x) for x in g.factor(len(configs) - 1)[1]} >= {O.DENSE, O.ONE}


# ----------------------------------------------------------------------------- radix base 4


def _base4_graph(configs):
    g = _vertex_graph(configs)
    assert g.set_base4() == 0
    return g


def test_base4_figure_example():
    """Appendix, Fig. base4: in group 4^0, neighbours 0 and 1 hold biases 2 and 3, so the group
    splits into value sub-groups 2 = {0} and 3 = {1}; the group's weight is 2 + 3 = 5 and a
    neighbour is drawn through group, sub-group, then uniformly inside the sub-group."""
    g = _base4_graph([(2, 3)])
    cnt, kd, sw = g.factor(0)
    # slot 3 i + v - 1: (i = 0, v = 2) -> slot 1, (i = 0, v = 3) -> slot 2
    assert [int(c) for c in cnt[:3]] == [0, 1, 1] and int(cnt[3:].sum()) == 0
    W = g.group_totals(0)
    assert int(W[1]) == 2 and int(W[2]) == 3 and int(W.sum()) == 5 == sw
    assert [Fraction(*g.factored_prob(0, i)) for i in range(2)] == [Fraction(2, 5), Fraction(3, 5)]


def test_base4_membership_by_digit_expansion():
    """Each edge sits in one sub-group per nonzero base-4 digit (counted here from the base-4
    numeral string), and the sub-group totals add up to the vertex's bias sum."""
    rng = np.random.default_rng(31)
    configs = [tuple(int(x) for x in rng.integers(1, 1 << 20, size=int(rng.integers(1, 9)))) for _ in range(200)]
    g = _base4_graph(configs)
    moffs, _ = g.members_all()
    for v, ws in enumerate(configs):
        nz = sum(sum(ch != "0" for ch in np.base_repr(w, 4)) for w in ws)
        assert int(moffs[32 * v + 32] - moffs[32 * v]) == nz
        assert int(g.group_totals(v).sum()) == sum(ws)
        cnt, _, _ = g.factor(v)
        positions = {k // 3 for k in range(32) if cnt[k]}
        assert max(positions) + 1 == max(len(np.base_repr(w, 4)) for w in ws)  # K = number of base-4 digits


def test_base4_theorem1_exact():
    configs = [c for d in (1, 2, 3) for c in itertools.product(range(1, 16), repeat=d)]
    rng = np.random.default_rng(32)
    configs += [tuple(int(x) for x in rng.integers(1, 1 << 20, size=int(rng.integers(4, 9)))) for _ in range(500)]
    configs += [tuple([1] * 9 + [2, 6]), tuple([3] * 30 + [12, 48]), tuple([7] * 3 + [1] * 40 + [64, 192])]
    g = _base4_graph(configs)
    kinds = set()
    for v, ws in enumerate(configs):
        kinds |= {int(x) for x in g.factor(v)[1]}
        s = sum(ws)
        for i, w in enumerate(ws):
            assert Fraction(*g.factored_prob(v, i)) == Fraction(w, s), (ws, i)
    assert {O.DENSE, O.ONE, O.SPARSE, O.REGULAR} <= kinds


def test_base4_validation_and_updates():
    g = O.Graph.from_edges(4, [(0, 1, (1 << 20) - 1)])
    assert g.set_base4() == 0
    assert g.apply(np.array([[0, 2, 1 << 20, 0]], dtype=np.uint32))[0] != 0
    rc, st = g.apply(np.array([[0, 2, 6, 0], [0, 1, 0, 1]], dtype=np.uint32))
    assert rc == 0 and st == (1, 1, 0)
    cnt, _, sw = g.factor(0)
    assert sw == 6 and int(cnt[1]) == 1 and int(cnt[3]) == 1 and int(cnt.sum()) == 2  # 6 = 2 + 1 * 4
    assert O.Graph.from_edges(2, [(0, 1, 1 << 20)]).set_base4() != 0
