"""Parity of the CUDA path's factorisation state with the oracle (bit-exact), through the C ABI.

After creation and after every update batch, the exported state must equal the
oracle's recomputation from scratch: edges (dst, bias, edge id) per vertex,
|G_k|, kinds, and every group's membership as a sorted set of edge ids; the
layout (member lists, inverted indexes, sparse lists) must satisfy its
invariants.  Update statistics (inserted, deleted, not_found) must match too.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from tests.conftest import golden
from tests.gpu_helpers import assert_state_matches

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


def make(B, G, host=False, **cfg):
    if host:
        return B.Graph(G.n, G.row_ptr, G.col, G.w, max_bits=G.max_bits, **cfg)
    return B.Graph(G.n, dev(G.row_ptr), dev(G.col), dev(G.w), max_bits=G.max_bits, **cfg)


def apply_both(g, og, rec, max_bits, stream=False):
    rec = np.ascontiguousarray(rec, dtype=np.uint32).reshape(-1, 4)
    if stream:
        st = g.stream_updates(dev(rec))
        tot = [0, 0, 0]
        for r in rec:
            rc, s = og.apply(r[None, :], max_bits)
            assert rc == 0
            tot = [a + b for a, b in zip(tot, s)]
        ost = tuple(tot)
    else:
        st = g.apply_updates(dev(rec))
        rc, ost = og.apply(rec, max_bits)
        assert rc == 0
    assert (st["inserted"], st["deleted"], st["not_found"]) == ost, (st, ost)
    return st


def test_create_parity_c1(B):
    wl = W.make_workload("c1")
    G = wl.graph
    g = make(B, G)
    assert_state_matches(g.export_state(), O.Graph(G.n, G.row_ptr, G.col, G.w))


def test_create_from_host_buffers_equals_device(B):
    wl = W.make_workload("c1")
    G = wl.graph
    a = make(B, G).export_state()
    b = make(B, G, host=True).export_state()
    for k in ("deg", "dst", "bias", "eid", "cnt", "kind", "members", "sp_list"):
        assert (a[k] == b[k]).all(), k


def test_c1_batch_parity(B):
    wl = W.make_workload("c1")
    G = wl.graph
    g = make(B, G)
    og = O.Graph(G.n, G.row_ptr, G.col, G.w)
    apply_both(g, og, wl.batches[0].records(), G.max_bits)
    assert_state_matches(g.export_state(), og)


def test_host_records_equal_device_records(B):
    wl = W.make_workload("c1")
    G = wl.graph
    g1, g2 = make(B, G), make(B, G)
    rec = wl.batches[0].records()
    s1 = g1.apply_updates(rec)
    s2 = g2.apply_updates(dev(rec))
    assert s1 == s2
    e1, e2 = g1.export_state(), g2.export_state()
    for k in ("deg", "dst", "bias", "eid", "cnt", "kind", "members", "sp_list"):
        assert (e1[k] == e2[k]).all(), k


def test_golden_update_semantics(B):
    gd = golden("update_semantics.json")
    og = O.Graph.from_edges(gd["n"], [tuple(e) for e in gd["initial"]])
    offs, dst, w, eid = og.edges()
    rp = offs.astype(np.uint64)
    g = B.Graph(gd["n"], dev(rp), dev(dst), dev(w), max_bits=32)
    for b in gd["batches"]:
        rec = np.array(b["records"], dtype=np.uint32)
        if b.get("status") == "invalid":
            with pytest.raises(B.BingoError) as ei:
                g.apply_updates(dev(rec))
            assert ei.value.status == B.E_INVALID
        else:
            st = g.apply_updates(dev(rec))
            assert [st["inserted"], st["deleted"], st["not_found"]] == b["stats"], b["why"]
            og.apply(rec, 32)
        ex = g.export_state()
        offs = np.concatenate([[0], np.cumsum(ex["deg"].astype(np.int64))])
        for v in range(gd["n"]):
            a, c = offs[v], offs[v + 1]
            got = sorted([[int(ex["dst"][j]), int(ex["bias"][j]), int(ex["eid"][j])] for j in range(a, c)],
                         key=lambda r: r[2])
            assert got == b["edges_after"].get(str(v), []), (b["why"], v)
        assert_state_matches(ex, og)


def test_invalid_batches_leave_state_unchanged(B):
    wl = W.make_workload("c1")
    G = wl.graph
    g = make(B, G)
    before = g.export_state()
    for bad in ([[0, G.n, 5, 0]], [[G.n, 0, 5, 1]], [[0, 1, 0, 0]], [[0, 1, 256, 0]], [[0, 1, 5, 3]]):
        rec = np.concatenate([wl.batches[0].records()[:10], np.array(bad, dtype=np.uint32)])
        with pytest.raises(B.BingoError) as ei:
            g.apply_updates(dev(rec))
        assert ei.value.status == B.E_INVALID
        with pytest.raises(B.BingoError):
            g.stream_updates(dev(rec))
    after = g.export_state()
    for k in ("deg", "dst", "bias", "eid", "cnt", "kind", "members", "sp_list"):
        assert (before[k] == after[k]).all(), k


def test_empty_batch_and_missing_deletes(B):
    wl = W.make_workload("c1")
    G = wl.graph
    g = make(B, G)
    og = O.Graph(G.n, G.row_ptr, G.col, G.w)
    st = g.apply_updates(np.zeros((0, 4), dtype=np.uint32))
    assert st["inserted"] == st["deleted"] == st["not_found"] == 0
    # deletions of edges that do not exist (self-loops never exist in the ER graph)
    rec = np.array([[v, v, 0, 1] for v in range(0, G.n, 7)], dtype=np.uint32)
    st = apply_both(g, og, rec, G.max_bits)
    assert st["not_found"] == len(rec) and st["deleted"] == 0
    assert_state_matches(g.export_state(), og)


def _stress_graph(seed, n=96, hubs=6, hub_deg=120, base_deg=6):
    """Small multigraph whose vertices cover every kind: hubs with mostly small biases and a few
    large ones (sparse and one-element groups), plain vertices, duplicates and isolated vertices."""
    rng = np.random.default_rng(seed)
    edges = []
    for v in range(n):
        d = hub_deg if v < hubs else (0 if v % 11 == 5 else base_deg + int(rng.integers(0, 8)))
        for _ in range(d):
            x = int(rng.integers(0, n))
            r = rng.random()
            w = int(rng.integers(1, 8)) if r < 0.85 else int(rng.integers(8, 1 << 12))
            edges.append((v, x, w))
    return O.Graph.from_edges(n, edges)


def _stress_batch(rng, og, n, size, wmax=1 << 12):
    offs, dst, w, eid = og.edges()
    rec = []
    for _ in range(size):
        op = rng.random()
        v = int(rng.integers(0, n)) if rng.random() < 0.6 else int(rng.integers(0, 6))
        if op < 0.45:
            x = int(rng.integers(0, n))
            b = int(rng.integers(1, 8)) if rng.random() < 0.8 else int(rng.integers(8, wmax))
            rec.append([v, x, b, 0])
        elif op < 0.9:
            a, c = int(offs[v]), int(offs[v + 1])
            x = int(dst[int(rng.integers(a, c))]) if c > a and rng.random() < 0.9 else int(rng.integers(0, n))
            rec.append([v, x, 0, 1])
        else:
            a, c = int(offs[v]), int(offs[v + 1])
            x = int(dst[int(rng.integers(a, c))]) if c > a else int(rng.integers(0, n))
            rec.append([v, x, int(rng.integers(1, wmax)), 2])
    return np.array(rec, dtype=np.uint32)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_random_batches_all_kinds(B, seed):
    og = _stress_graph(seed)
    offs, dst, w, eid = og.edges()
    n = og.n
    g = B.Graph(n, dev(offs.astype(np.uint64)), dev(dst), dev(w), max_bits=12)
    assert_state_matches(g.export_state(), og)
    rng = np.random.default_rng(100 + seed)
    conv_total = np.zeros((5, 5), dtype=np.int64)
    kinds_seen = set()
    for it in range(25):
        size = [1, 3, 17, 64, 300][it % 5]
        st = apply_both(g, og, _stress_batch(rng, og, n, size), 12)
        conv_total += np.array(st["conversions"])
        ex = g.export_state()
        kinds_seen |= set(np.unique(ex["kind"]).tolist())
        assert_state_matches(ex, og)
    assert {O.DENSE, O.ONE, O.SPARSE, O.REGULAR} <= kinds_seen
    assert conv_total.sum() > 0


def test_streaming_parity(B):
    og = _stress_graph(7)
    offs, dst, w, eid = og.edges()
    g = B.Graph(og.n, dev(offs.astype(np.uint64)), dev(dst), dev(w), max_bits=12)
    rng = np.random.default_rng(9)
    for it in range(4):
        apply_both(g, og, _stress_batch(rng, og, og.n, 200), 12, stream=True)
        assert_state_matches(g.export_state(), og)


def test_batch_after_a_stream_larger_than_its_capacity(B):
    """Streaming shares the batch pipeline's scratch buffers: a stream with more records than the
    captured batch capacity grows them, and the next batch must re-size and re-capture its pipeline
    instead of reusing the old buffers; batches, streams and batches again all match the oracle."""
    og = _stress_graph(5)
    offs, dst, w, eid = og.edges()
    g = B.Graph(og.n, dev(offs.astype(np.uint64)), dev(dst), dev(w), max_bits=12)
    rng = np.random.default_rng(17)
    apply_both(g, og, _stress_batch(rng, og, og.n, 300), 12)
    apply_both(g, og, _stress_batch(rng, og, og.n, 6000), 12, stream=True)
    apply_both(g, og, _stress_batch(rng, og, og.n, 300), 12)
    assert_state_matches(g.export_state(), og)
    g.check()


def test_streaming_large_vertices_use_block_teams(B):
    """Streamed records of vertices with at least 4,096 edges are applied by a whole block (after the
    warp pass over the smaller ones); duplicated edges, deletions of missing edges, set_bias and a
    vertex that crosses 4,096 edges inside the stream must all match the oracle, one record at a time."""
    n = 1 << 12
    rng = np.random.default_rng(21)
    edges = [(v, int(rng.integers(0, 64)), int(rng.integers(1, 1 << 10))) for v in range(3) for _ in range(6000)]
    edges += [(3, int(rng.integers(0, n)), int(rng.integers(1, 1 << 10))) for _ in range(4090)]
    edges += [(v, int(rng.integers(0, n)), int(rng.integers(1, 1 << 10))) for v in range(4, n) for _ in range(3)]
    og = O.Graph.from_edges(n, edges)
    offs, dst, w, eid = og.edges()
    g = B.Graph(n, dev(offs.astype(np.uint64)), dev(dst), dev(w), max_bits=10)
    for it in range(2):
        o_offs, o_dst, _, _ = og.edges()
        rec = []
        for _ in range(900):
            v = int(rng.integers(0, 4)) if rng.random() < 0.7 else int(rng.integers(4, n))
            a, c = int(o_offs[v]), int(o_offs[v + 1])
            op = rng.random()
            if op < 0.4:
                rec.append([v, int(rng.integers(0, 64 if v < 3 else n)), int(rng.integers(1, 1 << 10)), 0])
            elif op < 0.85:
                x = int(o_dst[int(rng.integers(a, c))]) if c > a and rng.random() < 0.9 else int(rng.integers(0, n))
                rec.append([v, x, 0, 1])
            else:
                x = int(o_dst[int(rng.integers(a, c))]) if c > a else int(rng.integers(0, n))
                rec.append([v, x, int(rng.integers(1, 1 << 10)), 2])
        apply_both(g, og, np.array(rec, dtype=np.uint32), 10, stream=True)
        assert_state_matches(g.export_state(), og)
    g.check()


def test_capacity_growth_and_emptying(B):
    # one vertex grows far past its capacity (every structure rebuilt), another loses every edge
    n = 4096
    edges = [(0, 1 + j, 1 + (j % 5)) for j in range(3)] + [(1, 2 + j, 3) for j in range(40)]
    og = O.Graph.from_edges(n, edges)
    offs, dst, w, eid = og.edges()
    g = B.Graph(n, dev(offs.astype(np.uint64)), dev(dst), dev(w), max_bits=16)
    rng = np.random.default_rng(3)
    ins = np.array([[0, int(rng.integers(0, n)), int(rng.integers(1, 1 << 16)), 0] for _ in range(5000)], np.uint32)
    apply_both(g, og, ins, 16)
    assert_state_matches(g.export_state(), og)
    dels = np.array([[1, 2 + j, 0, 1] for j in range(40)], np.uint32)
    apply_both(g, og, dels, 16)
    ex = g.export_state()
    assert ex["deg"][1] == 0 and (ex["kind"][1] == O.EMPTY).all()
    assert_state_matches(ex, og)
    # and refill it
    apply_both(g, og, np.array([[1, 7, 9, 0], [1, 7, 9, 0], [1, 8, 1, 0]], np.uint32), 16)
    assert_state_matches(g.export_state(), og)


def test_hub_segments_use_block_teams(B):
    # segments with > 256 updates or > 4096 slots run on a whole block; check them too
    n = 1 << 12
    rng = np.random.default_rng(11)
    edges = [(v, int(rng.integers(0, n)), int(rng.integers(1, 64))) for v in range(4) for _ in range(6000)]
    edges += [(v, int(rng.integers(0, n)), int(rng.integers(1, 64))) for v in range(4, n) for _ in range(3)]
    og = O.Graph.from_edges(n, edges)
    offs, dst, w, eid = og.edges()
    g = B.Graph(n, dev(offs.astype(np.uint64)), dev(dst), dev(w), max_bits=6)
    for it in range(3):
        rec = []
        for v in range(4):
            a, c = int(offs[v]), int(offs[v + 1])
            og_offs, og_dst, _, _ = og.edges()
            a, c = int(og_offs[v]), int(og_offs[v + 1])
            for _ in range(700):
                rec.append([v, int(og_dst[int(rng.integers(a, c))]), 0, 1])
            for _ in range(500):
                rec.append([v, int(rng.integers(0, n)), int(rng.integers(1, 64)), 0])
        rec = np.array(rec, dtype=np.uint32)
        rng.shuffle(rec)
        apply_both(g, og, rec, 6)
        assert_state_matches(g.export_state(), og)


def test_c2_scaled_batches(B):
    wl = W.make_workload("c2", scale=15, m=1 << 19, nbatch=4, batch=20000)
    G = wl.graph
    g = make(B, G)
    og = O.Graph(G.n, G.row_ptr, G.col, G.w)
    assert_state_matches(g.export_state(), og)
    for b in wl.batches:
        apply_both(g, og, b.records(), G.max_bits)
        assert_state_matches(g.export_state(), og)


def test_c2_full_size_first_batches(B):
    """BASELINE sizes of the RMAT-20 workload (16M edges, batches of 10^5), as bench.py runs it."""
    wl = W.make_workload("c2", nbatch=2)
    G = wl.graph
    g = make(B, G)
    og = O.Graph(G.n, G.row_ptr, G.col, G.w)
    assert_state_matches(g.export_state(), og)
    for b in wl.batches:
        apply_both(g, og, b.records(), G.max_bits)
    assert_state_matches(g.export_state(), og)


def test_pool_exhaustion_rejects_batch_unchanged(B):
    """A pool sized to the created state leaves no room for growth: a batch that grows vertices must be
    rejected with BINGO_E_OOM before any change, and the streaming path must stop cleanly."""
    wl = W.make_workload("c1")
    G = wl.graph
    probe = make(B, G)
    used = probe.export_state()["sizes"]["pool_words_used"]
    probe.close()
    g = make(B, G, pool_words=int(used) + 64)
    before = g.export_state()
    rng = np.random.default_rng(1)
    grow = np.array([[v, int(rng.integers(0, G.n)), 1 + int(rng.integers(0, 200)), 0]
                     for v in range(0, 64) for _ in range(40)], dtype=np.uint32)
    with pytest.raises(B.BingoError) as ei:
        g.apply_updates(dev(grow))
    assert ei.value.status == B.E_OOM
    after = g.export_state()
    for k in ("deg", "dst", "bias", "eid", "cnt", "kind", "members", "sp_list"):
        assert (before[k] == after[k]).all(), k
    og = O.Graph(G.n, G.row_ptr, G.col, G.w)
    assert_state_matches(after, og)  # still the created state, exactly
    import torch

    paths = torch.empty((64, 11), dtype=torch.int32, device="cuda")
    plen = torch.empty(64, dtype=torch.int32, device="cuda")
    g.walk(dev(np.arange(64, dtype=np.uint32)), [B.policy(B.DEEPWALK, 10)], 3, 11, paths, plen)
    g.check()
    with pytest.raises(B.BingoError) as ei:
        g.stream_updates(dev(grow))
    assert ei.value.status == B.E_OOM
    ex = g.export_state()  # whatever streamed before the stop is complete and consistent
    from tests.gpu_helpers import check_layout_invariants
    check_layout_invariants(ex)


def test_baseline_all_regular_parity_and_memory(B):
    """The BS baseline of the group-adaption ablation (Section 6.2): every nonempty group regular.
    Bit-exact against the oracle's BS mode through batches and streaming; group adaption (Eq. group)
    needs less memory for group structures on the same graph."""
    og = _stress_graph(12)
    offs, dst, w, eid = og.edges()
    bs = B.Graph(og.n, dev(offs.astype(np.uint64)), dev(dst), dev(w), max_bits=12, all_regular=1)
    ga = B.Graph(og.n, dev(offs.astype(np.uint64)), dev(dst), dev(w), max_bits=12)
    ex = bs.export_state()
    assert_state_matches(ex, og, O.ALL_REGULAR, 0)
    assert set(np.unique(ex["kind"]).tolist()) == {O.EMPTY, O.REGULAR}
    mem_bs, mem_ga = bs.memory_report(), ga.memory_report()
    assert mem_ga["regular_groups"] + mem_ga["sparse_groups"] < mem_bs["regular_groups"]
    rng = np.random.default_rng(77)
    for it in range(8):
        rec = _stress_batch(rng, og, og.n, [1, 17, 300, 64][it % 4])
        if it % 2:
            apply_both(bs, og, rec, 12, stream=True)
        else:
            apply_both(bs, og, rec, 12)
        assert_state_matches(bs.export_state(), og, O.ALL_REGULAR, 0)


def test_radix_base4_parity(B):
    """Radix base 4 (Appendix): value sub-groups per base-4 digit, in slots 3 i + v - 1.  Bit-exact
    against the oracle's base-4 mode through creation, batches and streaming records."""
    og = _stress_graph(13)
    assert og.set_base4() == 0
    offs, dst, w, eid = og.edges()
    g = B.Graph(og.n, dev(offs.astype(np.uint64)), dev(dst), dev(w), max_bits=12, radix_base=4)
    ex = g.export_state()
    assert_state_matches(ex, og, base4=True)
    assert set(np.unique(ex["kind"]).tolist()) >= {O.DENSE, O.ONE, O.REGULAR}
    rng = np.random.default_rng(88)
    for it in range(8):
        rec = _stress_batch(rng, og, og.n, [1, 17, 300, 64][it % 4])
        apply_both(g, og, rec, 12, stream=bool(it % 2))
        assert_state_matches(g.export_state(), og, base4=True)
    with pytest.raises(B.BingoError):
        B.Graph(og.n, dev(offs.astype(np.uint64)), dev(dst), dev(np.full_like(w, 1 << 20)), radix_base=4)


def test_hub_prepass_deletions(B):
    """A hub past the grid-wide pre-pass threshold (d >= 2^16): deletions of duplicated edges, repeated
    deletions of one destination, deletions of edges inserted in the same batch and misses, all
    resolved to the earliest live copy as the oracle does."""
    n = 4096
    rng = np.random.default_rng(91)
    hub_d = 70000
    edges = [(0, int(x), int(w)) for x, w in zip(rng.integers(1, 2000, hub_d), rng.integers(1, 1 << 10, hub_d))]
    edges += [(1 + (j % 50), int(rng.integers(0, n)), 3) for j in range(2000)]
    og = O.Graph.from_edges(n, edges)
    offs, dst, w, eid = og.edges()
    g = B.Graph(n, dev(offs.astype(np.uint64)), dev(dst), dev(w), max_bits=10)
    for it in range(4):
        rec = []
        hub_dst = dst[int(offs[0]):int(offs[1])]
        for _ in range(400):  # deletions of live hub edges (destinations repeat: duplicates exist)
            rec.append([0, int(hub_dst[int(rng.integers(0, len(hub_dst)))]), 0, 1])
        for _ in range(100):  # insert-then-delete in one batch, and misses
            x = int(rng.integers(2000, 3000))
            rec.append([0, x, int(rng.integers(1, 1 << 10)), 0])
            rec.append([0, x, 0, 1])
            rec.append([0, int(rng.integers(3000, n)), 0, 1])
        for _ in range(300):
            rec.append([0, int(rng.integers(1, 2000)), int(rng.integers(1, 1 << 10)), 0])
        rec = np.array(rec, dtype=np.uint32)
        rec = rec[rng.permutation(len(rec))]
        st = apply_both(g, og, rec, 10)
        assert st["not_found"] > 0 and st["deleted"] > 0
        offs, dst, w, eid = og.edges()
        assert_state_matches(g.export_state(), og)


def test_update_autotune_applies_slices_in_order(B):
    """bingo_autotune_updates applies the records as ten consecutive slices (five settings, two
    rounds) and keeps one of the candidate update_chunk settings; the state equals the oracle's
    after the same slices."""
    og = _stress_graph(21)
    offs, dst, w, eid = og.edges()
    g = B.Graph(og.n, dev(offs.astype(np.uint64)), dev(dst), dev(w), max_bits=12)
    rng = np.random.default_rng(22)
    rec = _stress_batch(rng, og, og.n, 1003)
    st, cfg = g.autotune_updates(dev(rec))
    assert cfg.update_chunk in (1024, 2048, 4096, 8192, 16384)
    sl = len(rec) // 10
    tot = [0, 0, 0]
    for k in range(10):
        part = rec[k * sl: (k + 1) * sl] if k < 9 else rec[9 * sl:]
        rc, s = og.apply(part, 12)
        assert rc == 0
        tot = [a + b for a, b in zip(tot, s)]
    assert (st["inserted"], st["deleted"], st["not_found"]) == tuple(tot)
    assert_state_matches(g.export_state(), og)
    apply_both(g, og, _stress_batch(rng, og, og.n, 200), 12)  # the kept setting serves later batches
    assert_state_matches(g.export_state(), og)


def test_adaption_autotune_choice_parity_and_budget(B):
    """bingo_autotune_adaption returns one of its (alpha, beta) candidates, in exactly the state a plain
    create with that pair gives (oracle parity under the chosen thresholds, before and after a batch);
    only candidates within the state budget can be chosen, and a budget below every candidate is
    BINGO_E_OOM."""
    wl = W.make_workload("c2", scale=14, m=1 << 18, nbatch=1, batch=1000)
    G = wl.graph
    starts = W.walk_starts(G.n, 1 << 15, 0)
    og = O.Graph(G.n, G.row_ptr, G.col, G.w)
    mem = {}
    for a in (20, 40, 70, 100):
        for b in (0, 10):
            g = make(B, G, alpha_pct=a, beta_pct=b)
            r = g.memory_report()
            mem[(a, b)] = r["adjacency"] + r["vertex_records"] + r["regular_groups"] + r["sparse_groups"]
            g.close()
    assert len(set(mem.values())) > 1  # the candidates really differ in memory
    t = B.Graph.tuned(G.n, dev(G.row_ptr), dev(G.col), dev(G.w), dev(starts), 20, max_bits=G.max_bits)
    pick = (t.cfg.alpha_pct, t.cfg.beta_pct)
    assert pick in mem
    assert_state_matches(t.export_state(), og, alpha=pick[0], beta=pick[1])
    apply_both(t, og, wl.batches[0].records(), G.max_bits)
    assert_state_matches(t.export_state(), og, alpha=pick[0], beta=pick[1])
    t.close()
    budget = min(mem.values())  # host inputs this time
    t = B.Graph.tuned(G.n, G.row_ptr, G.col, G.w, starts, 20, state_budget_bytes=budget, max_bits=G.max_bits)
    assert mem[(t.cfg.alpha_pct, t.cfg.beta_pct)] <= budget
    t.close()
    with pytest.raises(B.BingoError) as ei:
        B.Graph.tuned(G.n, dev(G.row_ptr), dev(G.col), dev(G.w), dev(starts), 20, state_budget_bytes=budget - 1,
                      max_bits=G.max_bits)
    assert ei.value.status == B.E_OOM
