"""Walks on the CUDA path, through the C ABI, against the oracle.

Statistical parity: one-step transition frequencies at >= 10^6 samples must
agree with the oracle's w / sum w (TV <= 0.01 and chi-square p > 1e-3;
neighbours are binned in edge-id order with exact bin masses, into <= 1,000
bins for chi-square and <= 256 bins for TV, whose sampling noise alone grows
as sqrt(bins / samples)).
Every step of every walk must be a live edge of the oracle graph at that
epoch.  Bit-exact GPU-vs-GPU: paths do not depend on the team width, the
launch form (persistent / stepwise) or on other requests in a merged launch.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from tests.conftest import golden
from tests.gpu_helpers import assert_steps_live, edge_keys
from tests.stats import binned, chisq_p, tv

pytestmark = pytest.mark.gpu
N_SAMPLES = 1_000_000


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


def run_walk(B, g, starts, policies, seed, stride, lengths=None, pids=None, mode=0):
    import torch

    n = len(starts)
    paths = torch.empty((n, stride), dtype=torch.int32, device="cuda")
    plen = torch.empty(n, dtype=torch.int32, device="cuda")
    g.walk(dev(starts), policies, seed, stride, paths, plen,
           lengths=None if lengths is None else dev(lengths),
           policy_ids=None if pids is None else dev(pids), mode=mode)
    g.check()
    return paths.cpu().numpy().view(np.uint32), plen.cpu().numpy().view(np.uint32)


def graph_of(B, G, **cfg):
    return B.Graph(G.n, dev(G.row_ptr), dev(G.col), dev(G.w), max_bits=G.max_bits, **cfg)


def one_step_check(B, g, og, v, seed):
    """10^6 one-step samples from v against the oracle's w / sum w (duplicates merged)."""
    offs, dst, w, _ = og.edges()
    a, c = int(offs[v]), int(offs[v + 1])
    d = dst[a:c].astype(np.int64)
    ww = w[a:c].astype(np.float64)
    uniq, inv = np.unique(d, return_inverse=True)
    probs = np.bincount(inv, weights=ww)
    starts = np.full(N_SAMPLES, v, dtype=np.uint32)
    paths, plen = run_walk(B, g, starts, [B.policy(B.DEEPWALK, 1)], seed, 2)
    assert (plen == 2).all()
    got = paths[:, 1].astype(np.int64)
    pos = np.searchsorted(uniq, got)
    assert (uniq[np.minimum(pos, len(uniq) - 1)] == got).all(), "sampled a non-neighbour"
    counts = np.bincount(pos, minlength=len(uniq)).astype(np.float64)
    # chi-square on up to 1,000 bins; TV on up to 256 bins, because multinomial noise alone gives
    # E[TV] ~ 0.5 sqrt(2K / (pi N)): 0.0126 at K = 1,000 and N = 10^6, 0.0064 at K = 256
    cb, pb = binned(counts, probs, 1000)
    p = chisq_p(cb, pb)
    tb, tpb = binned(counts, probs, 256)
    t = tv(tb, tpb)
    assert t <= 0.01, (v, t)
    assert p > 1e-3, (v, p)
    return t, p


def pick_vertices(og, ex_kind, want):
    """Distinct vertices: for each requested kind, the highest-degree and a median-degree vertex
    that have a group of that kind."""
    offs, _, _, _ = og.edges()
    deg = np.diff(offs.astype(np.int64))
    out = []
    for kd in want:
        cand = np.nonzero((ex_kind == kd).any(axis=1) & (deg > 0))[0]
        cand = np.array([c for c in cand if int(c) not in out], dtype=np.int64)
        if len(cand):
            order = cand[np.argsort(deg[cand])]
            out.append(int(order[-1]))
            if len(order) > 2:
                out.append(int(order[len(order) // 2]))
    return sorted(set(out))


def test_one_step_distribution_c1(B):
    wl = W.make_workload("c1")
    G = wl.graph
    g = graph_of(B, G)
    og = O.Graph(G.n, G.row_ptr, G.col, G.w)
    for i, v in enumerate((0, 333, 1023)):
        one_step_check(B, g, og, v, 10 + i)


def test_one_step_distribution_every_kind_and_after_updates(B):
    wl = W.make_workload("c2", scale=16, m=1 << 20, nbatch=2, batch=50000)
    G = wl.graph
    g = graph_of(B, G)
    og = O.Graph(G.n, G.row_ptr, G.col, G.w)
    kinds = g.export_state()["kind"]
    vs = pick_vertices(og, kinds, [O.DENSE, O.ONE, O.SPARSE, O.REGULAR])
    assert len(vs) >= 3
    for i, v in enumerate(vs):
        one_step_check(B, g, og, v, 100 + i)
    for b in wl.batches:
        rec = b.records()
        g.apply_updates(dev(rec))
        og.apply(rec, G.max_bits)
    touched = np.unique(wl.batches[-1].src)
    offs, _, _, _ = og.edges()
    deg = np.diff(offs.astype(np.int64))
    t = touched[np.argsort(-deg[touched])][:3]
    for i, v in enumerate(t):
        one_step_check(B, g, og, int(v), 200 + i)


def test_hub_one_step_binned(B):
    n = 1 << 12
    rng = np.random.default_rng(4)
    d = 30000
    edges = [(0, int(rng.integers(0, n)), int(rng.integers(1, 1 << 20))) for _ in range(d)]
    edges += [(v, int(rng.integers(0, n)), 1) for v in range(1, n) for _ in range(2)]
    og = O.Graph.from_edges(n, edges)
    offs, dst, w, _ = og.edges()
    g = B.Graph(n, dev(offs.astype(np.uint64)), dev(dst), dev(w), max_bits=20)
    one_step_check(B, g, og, 0, 77)


def test_group_selection_law_at_a_hub(B):
    """Group selection on its own (Eq. group_prob): with power-of-two biases each edge lies in exactly
    one group, and with distinct destinations each sampled neighbour names its edge, so 10^6 one-step
    samples from a hub whose groups take every kind (dense, regular, sparse, one-element) give the
    group frequencies, which must match W_k / sum_j W_j, W_k = 2^k |G_k| (TV <= 0.01, chi-square
    p > 1e-3; at most 32 categories)."""
    n = 1 << 15
    rng = np.random.default_rng(12)
    d = 20000
    ks = np.concatenate([np.zeros(9000), np.full(4000, 3), rng.integers(5, 16, size=d - 13001), [19]]).astype(np.int64)
    rng.shuffle(ks)
    dsts = rng.permutation(n)[:d]
    edges = [(0, int(x), 1 << int(k)) for x, k in zip(dsts, ks)] + [(v, (v + 1) % n, 1) for v in range(1, n)]
    og = O.Graph.from_edges(n, edges)
    offs, dst, w, _ = og.edges()
    g = B.Graph(n, dev(offs.astype(np.uint64)), dev(dst), dev(w), max_bits=20)
    ex = g.export_state()
    assert {O.DENSE, O.REGULAR, O.SPARSE, O.ONE} <= set(ex["kind"][0][ex["cnt"][0] > 0].tolist())
    paths, plen = run_walk(B, g, np.zeros(N_SAMPLES, np.uint32), [B.policy(B.DEEPWALK, 1)], 21, 2)
    assert (plen == 2).all()
    group_of = np.full(n, -1, dtype=np.int64)
    group_of[dsts] = ks
    got = group_of[paths[:, 1].astype(np.int64)]
    assert (got >= 0).all(), "sampled a non-neighbour"
    cnt = np.bincount(ks, minlength=20).astype(np.float64)
    W_k = cnt * np.exp2(np.arange(20))
    live = cnt > 0
    counts = np.bincount(got, minlength=20).astype(np.float64)[live]
    probs = (W_k / W_k.sum())[live]
    assert tv(counts, probs) <= 0.01
    assert chisq_p(counts, probs) > 1e-3


@pytest.mark.parametrize("name", ["c1", "c2s"])
def test_every_step_is_a_live_edge(B, name):
    wl = W.make_workload("c1") if name == "c1" else W.make_workload("c2", scale=15, m=1 << 19, nbatch=2, batch=20000)
    G = wl.graph
    g = graph_of(B, G)
    og = O.Graph(G.n, G.row_ptr, G.col, G.w)
    nw = min(G.n, 1 << 15)
    starts = W.walk_starts(G.n, nw, 0)
    pol = B.policy(B.DEEPWALK, wl.length)
    paths, plen = run_walk(B, g, starts, [pol], 0, wl.length + 1)
    assert (paths[:, 0] == starts).all()
    assert_steps_live(og, paths, plen)
    for ep, b in enumerate(wl.batches):
        rec = b.records()
        g.apply_updates(dev(rec))
        og.apply(rec, G.max_bits)
        paths, plen = run_walk(B, g, starts, [pol], ep + 1, wl.length + 1)
        assert_steps_live(og, paths, plen)


def test_c2_full_size_walk_in_the_bench_launch(B):
    """The bench workload at full size (RMAT-20, 2^24 edges, 2^20 DeepWalk walkers x 80) after one
    10^5-update batch, in the launch bench.py times (tuned shape, persistent form, no padding):
    every step is a live edge of the oracle graph, lengths are in range and the start is entry 0;
    and the one-step law at the highest-degree vertex (binned) holds at this size."""
    import torch

    wl = W.make_workload("c2", nbatch=1)
    G = wl.graph
    g = graph_of(B, G)
    og = O.Graph(G.n, G.row_ptr, G.col, G.w)
    rec = wl.batches[0].records()
    g.apply_updates(dev(rec))
    og.apply(rec, G.max_bits)
    starts = W.walk_starts(G.n, wl.nwalkers, wl.walk_seed)
    ds = dev(starts)
    g.autotune(ds, wl.length)
    stride = wl.length + 1
    paths = torch.full((wl.nwalkers, stride), -3, dtype=torch.int32, device="cuda")
    plen = torch.zeros(wl.nwalkers, dtype=torch.int32, device="cuda")
    g.walk(ds, [B.policy(B.DEEPWALK, wl.length)], 1, stride, paths, plen, mode=B.WALK_PERSISTENT | B.WALK_NO_PAD)
    g.check()
    p = paths.cpu().numpy().view(np.uint32)
    l = plen.cpu().numpy().view(np.uint32)
    assert (l >= 1).all() and (l <= stride).all() and (p[:, 0] == starts).all()
    assert int((l.astype(np.int64) - 1).sum()) > 20_000_000  # the walk really ran at scale
    assert_steps_live(og, p, l, padded=False)
    offs, _, _, _ = og.edges()
    hub = int(np.argmax(np.diff(offs.astype(np.int64))))
    one_step_check(B, g, og, hub, 9)


def _mixed_policies(B):
    return [B.policy(B.DEEPWALK, 20), B.policy(B.PPR, 30, 0.15), B.policy(B.NODE2VEC, 25, n2v_pq=(2.0, 0.5))]


def test_paths_independent_of_team_width_and_launch_form(B):
    wl = W.make_workload("c2", scale=14, m=1 << 18, nbatch=1, batch=4000)
    G = wl.graph
    g = graph_of(B, G)
    nw = 20000
    starts = W.walk_starts(G.n, nw, 1)
    pids = (np.arange(nw) % 3).astype(np.uint8)
    pols = _mixed_policies(B)
    ref = None
    for lanes in (1, 4, 32):
        for wpb, regv in ((4, 0), (8, 0), (16, 0), (4, 1), (8, 1)):
            g.set_walk_config(lanes, wpb, 0, regv)
            res = run_walk(B, g, starts, pols, 42, 31, pids=pids)
            if ref is None:
                ref = res
            assert (res[0] == ref[0]).all() and (res[1] == ref[1]).all(), (lanes, wpb, regv)
    step = run_walk(B, g, starts, pols, 42, 31, pids=pids, mode=B.WALK_STEPWISE)
    assert (step[0] == ref[0]).all() and (step[1] == ref[1]).all()
    other = run_walk(B, g, starts, pols, 43, 31, pids=pids)
    assert (other[0] != ref[0]).any()
    og = O.Graph(G.n, G.row_ptr, G.col, G.w)
    assert_steps_live(og, ref[0], ref[1])


def test_ppr_length_distribution(B):
    n = 64
    edges = [(v, (v + 1) % n, 1 + v % 5) for v in range(n)] + [(v, (v * 7 + 3) % n, 2) for v in range(n)]
    og = O.Graph.from_edges(n, edges)
    offs, dst, w, _ = og.edges()
    g = B.Graph(n, dev(offs.astype(np.uint64)), dev(dst), dev(w), max_bits=8)
    s_u32, cap = 644245094, 30
    paths, plen = run_walk(B, g, W.walk_starts(n, N_SAMPLES, 3), [B.policy(B.PPR, cap, s_u32)], 5, cap + 1)
    steps = plen.astype(np.int64) - 1
    counts = np.bincount(steps, minlength=cap + 1)
    s = s_u32 / 2 ** 32
    probs = np.array([(1 - s) ** l * s for l in range(cap)] + [(1 - s) ** cap])
    assert tv(counts, probs) < 0.01
    assert chisq_p(counts, probs) > 1e-3


def _n2v_two_step(B, g, accept, seed):
    starts = np.zeros(N_SAMPLES, dtype=np.uint32)
    pol = B.policy(B.NODE2VEC, 2)
    for i in range(3):
        pol.n2v_accept[i] = accept[i]
    return run_walk(B, g, starts, [pol], seed, 3)


def test_node2vec_tiny_closed_form(B):
    gd = golden("node2vec_tiny.json")
    og = O.Graph.from_edges(gd["n"], [tuple(e) for e in gd["edges"]])
    offs, dst, w, _ = og.edges()
    g = B.Graph(gd["n"], dev(offs.astype(np.uint64)), dev(dst), dev(w), max_bits=8)
    paths, plen = _n2v_two_step(B, g, gd["accept_u32"], 9)
    assert (plen == 3).all()
    tp = gd["two_step_paths_from_0"]
    keys = {tuple(p): i for i, p in enumerate(tp["paths"])}
    code = paths[:, 1].astype(np.int64) * 16 + paths[:, 2].astype(np.int64)
    counts = np.zeros(len(keys))
    for (a, b, c), i in keys.items():
        counts[i] = (code == b * 16 + c).sum()
    assert counts.sum() == N_SAMPLES
    probs = np.array(tp["prob_num"], float) / tp["prob_den"]
    assert tv(counts, probs) < 0.01 and chisq_p(counts, probs) > 1e-3


def test_node2vec_edge_index_follows_updates(B):
    gd = golden("node2vec_tiny.json")
    og = O.Graph.from_edges(gd["n"], [tuple(e) for e in gd["edges"]])
    offs, dst, w, _ = og.edges()
    g = B.Graph(gd["n"], dev(offs.astype(np.uint64)), dev(dst), dev(w), max_bits=8)
    _n2v_two_step(B, g, gd["accept_u32"], 1)  # builds the edge index
    # delete 0 -> 2 and add 0 -> 3: from 1 after 0, neighbour 2 becomes distance 2 and 3 distance 1
    rec = np.array([[0, 2, 0, 1], [0, 3, 1, 0]], dtype=np.uint32)
    g.apply_updates(dev(rec))
    og.apply(rec, 8)
    paths, plen = _n2v_two_step(B, g, gd["accept_u32"], 2)
    assert (paths[:, 1] == 1).sum() + (paths[:, 1] == 3).sum() == N_SAMPLES
    sel = paths[:, 1] == 1
    wts = og.n2v_weights(0, 1, gd["accept_u32"]).astype(np.float64)
    o2, d2, _, _ = og.edges()
    nb = d2[o2[1]:o2[2]].astype(np.int64)
    counts = np.array([(paths[sel, 2] == x).sum() for x in nb], dtype=np.float64)
    assert tv(counts, wts) < 0.01 and chisq_p(counts, wts) > 1e-3


def test_node2vec_edge_index_after_repeated_and_missing_deletions(B):
    """The edge index counts live copies: a batch that deletes the one copy of 0 -> 2 twice and deletes an
    edge that does not exist must leave 0 -> 2 absent (count 0, not one below it) and the rest unchanged,
    so from 1 after 0 the neighbour 2 is at distance 2, as the oracle's Eq. node2vec weights say."""
    gd = golden("node2vec_tiny.json")
    og = O.Graph.from_edges(gd["n"], [tuple(e) for e in gd["edges"]])
    offs, dst, w, _ = og.edges()
    g = B.Graph(gd["n"], dev(offs.astype(np.uint64)), dev(dst), dev(w), max_bits=8)
    _n2v_two_step(B, g, gd["accept_u32"], 1)  # builds the edge index
    assert (0, 2) in {(int(a), int(b)) for a, b, _ in gd["edges"]}
    missing = next(x for x in range(gd["n"]) if x not in {int(b) for a, b, _ in gd["edges"] if int(a) == 1})
    rec = np.array([[0, 2, 0, 1], [0, 2, 0, 1], [1, missing, 0, 1]], dtype=np.uint32)
    st = g.apply_updates(dev(rec))
    rc, ost = og.apply(rec, 8)
    assert rc == 0 and (st["deleted"], st["not_found"]) == (ost[1], ost[2]) == (1, 2)
    paths, plen = _n2v_two_step(B, g, gd["accept_u32"], 2)
    sel = paths[:, 1] == 1
    assert sel.sum() > 0
    wts = og.n2v_weights(0, 1, gd["accept_u32"]).astype(np.float64)
    o2, d2, _, _ = og.edges()
    nb = d2[o2[1]:o2[2]].astype(np.int64)
    counts = np.array([(paths[sel, 2] == x).sum() for x in nb], dtype=np.float64)
    assert tv(counts, wts) < 0.01 and chisq_p(counts, wts) > 1e-3


def test_padding_flag_and_host_buffers(B):
    wl = W.make_workload("c1")
    G = wl.graph
    g = graph_of(B, G)
    starts = W.walk_starts(G.n, 4096, 0)
    pol = [B.policy(B.PPR, 40, 0.2)]
    p1, l1 = run_walk(B, g, starts, pol, 7, 41)
    # host numpy buffers through the same entry point
    p2 = np.zeros((4096, 41), dtype=np.uint32)
    l2 = np.zeros(4096, dtype=np.uint32)
    g.walk(starts, pol, 7, 41, p2, l2)
    assert (p1 == p2).all() and (l1 == l2).all()
    # no-pad: entries beyond path_len untouched
    p3 = np.full((4096, 41), 0x12345678, dtype=np.uint32)
    g.walk(starts, pol, 7, 41, p3, l2, mode=B.WALK_NO_PAD)
    idx = np.arange(41)[None, :] >= l1[:, None].astype(np.int64)
    assert (p3[idx] == 0x12345678).all() and (p3[~idx] == p1[~idx]).all()


def test_host_buffer_walk_in_chunks_equals_device_walk(B):
    """Host-output walks of >= 2^17 walkers download id-ordered chunks of rows while the walk runs,
    each as soon as its last walker finished; every row must equal the device-buffer walk."""
    import torch

    wl = W.make_workload("c2", scale=14, m=1 << 18, nbatch=1, batch=1000)
    G = wl.graph
    g = graph_of(B, G)
    n, stride = 300_001, 23  # 19 chunks of 2^14 walkers, the last one ragged (5,089)
    starts = W.walk_starts(G.n, n, 5)
    lengths = (np.arange(n) % 23).astype(np.uint32)  # includes zero-length walks
    pids = (np.arange(n) % 2).astype(np.uint8)
    pols = [B.policy(B.DEEPWALK, 22), B.policy(B.PPR, 22, 0.15)]
    p1, l1 = run_walk(B, g, starts, pols, 9, stride, lengths=lengths, pids=pids)
    assert (l1 == np.minimum(lengths, 22) + 1).sum() > n // 4  # many walks run to their length
    # pageable host inputs and outputs
    p2 = np.zeros((n, stride), np.uint32)
    l2 = np.zeros(n, np.uint32)
    g.walk(starts, pols, 9, stride, p2, l2, lengths=lengths, policy_ids=pids)
    assert (p2 == p1).all() and (l2 == l1).all()
    # pinned host outputs, device inputs
    p3 = torch.zeros((n, stride), dtype=torch.int32).pin_memory()
    l3 = torch.zeros(n, dtype=torch.int32).pin_memory()
    g.walk(dev(starts), pols, 9, stride, p3, l3, lengths=dev(lengths), policy_ids=dev(pids))
    assert (p3.numpy().view(np.uint32) == p1).all() and (l3.numpy().view(np.uint32) == l1).all()
    # device paths, host lengths only
    p4 = torch.zeros((n, stride), dtype=torch.int32, device="cuda")
    l4 = np.zeros(n, np.uint32)
    g.walk(starts, pols, 9, stride, p4, l4, lengths=lengths, policy_ids=pids)
    assert (p4.cpu().numpy().view(np.uint32) == p1).all() and (l4 == l1).all()
    # no padding: entries beyond path_len keep the caller's values through the chunked round trip
    p5 = np.full((n, stride), 0x12345678, dtype=np.uint32)
    g.walk(starts, pols, 9, stride, p5, l2, lengths=lengths, policy_ids=pids, mode=B.WALK_NO_PAD)
    idx = np.arange(stride)[None, :] >= l1[:, None].astype(np.int64)
    assert (p5[idx] == 0x12345678).all() and (p5[~idx] == p1[~idx]).all()
    g.check()


def test_bounded_rejection_loop_reports_timeout(B):
    """Every device loop is bounded.  A node2vec policy that accepts no candidate (all thresholds 0)
    exhausts the rejection loop of every second step: the walk ends after its first-order step, the
    device status reads BINGO_E_TIMEOUT through bingo_check, the status is then clear, and the graph
    keeps walking correctly."""
    import torch

    wl = W.make_workload("c1")
    G = wl.graph
    g = graph_of(B, G)
    og = O.Graph(G.n, G.row_ptr, G.col, G.w)
    pol = B.policy(B.NODE2VEC, 5, n2v_pq=(2.0, 0.5))
    for i in range(3):
        pol.n2v_accept[i] = 0
    n = 256
    starts = W.walk_starts(G.n, n, 0)
    paths = torch.empty((n, 6), dtype=torch.int32, device="cuda")
    plen = torch.empty(n, dtype=torch.int32, device="cuda")
    g.walk(dev(starts), [pol], 1, 6, paths, plen)
    with pytest.raises(B.BingoError) as ei:
        g.check()
    assert ei.value.status == B.E_TIMEOUT
    p = paths.cpu().numpy().view(np.uint32)
    l = plen.cpu().numpy().view(np.uint32)
    assert (l <= 2).all() and (l == 2).sum() > n // 2  # the first-order step, then the loop gave up
    assert_steps_live(og, p, l)
    g.check()  # the status was cleared
    p2, l2 = run_walk(B, g, starts, [B.policy(B.DEEPWALK, 5)], 2, 6)
    assert (l2 == 6).all()
    assert_steps_live(og, p2, l2)


def test_invalid_walk_arguments(B):
    wl = W.make_workload("c1")
    G = wl.graph
    g = graph_of(B, G)
    with pytest.raises(B.BingoError):  # max_len does not fit the stride
        run_walk(B, g, np.zeros(4, np.uint32), [B.policy(B.DEEPWALK, 80)], 0, 10)
    with pytest.raises(B.BingoError) as ei:  # start vertex out of range (latched on the device)
        run_walk(B, g, np.array([0, G.n + 5], np.uint32), [B.policy(B.DEEPWALK, 3)], 0, 4)
    assert ei.value.status == B.E_INVALID
    # zero-length walks and dead ends
    paths, plen = run_walk(B, g, np.array([1, 2], np.uint32), [B.policy(B.DEEPWALK, 0)], 0, 1)
    assert (plen == 1).all() and (paths[:, 0] == [1, 2]).all()


def test_autotune_keeps_results(B):
    wl = W.make_workload("c2", scale=14, m=1 << 18, nbatch=1, batch=1000)
    G = wl.graph
    g = graph_of(B, G)
    starts = W.walk_starts(G.n, 50000, 0)
    pol = [B.policy(B.DEEPWALK, 30)]
    before = run_walk(B, g, starts, pol, 3, 31)
    cfg = g.autotune(dev(starts), 30)
    assert cfg.lanes_per_walker in (1, 4, 32)
    after = run_walk(B, g, starts, pol, 3, 31)
    assert (before[0] == after[0]).all()


def test_server_results_same_alone_and_in_the_mix(B):
    import ctypes

    wl = W.make_workload("c2", scale=14, m=1 << 18, nbatch=1, batch=2000)
    G = wl.graph
    g = graph_of(B, G)
    L = B.load()
    pol = B.policy(B.PPR, 40, 0.15)
    reqs = [(W.walk_starts(G.n, int(nw), 10 + i), 1000 + i) for i, nw in enumerate([1, 37, 500, 4096, 9])]

    def serve(subset, updates=None):
        h = ctypes.c_void_p()
        cfg = B.bingo_server_config()
        assert L.bingo_server_create(g.h, ctypes.byref(cfg), ctypes.byref(h)) == 0
        if updates is not None:
            ep = ctypes.c_uint64()
            assert L.bingo_server_submit_updates(h, updates.ctypes.data, len(updates), ctypes.byref(ep)) == 0
            assert L.bingo_server_drain(h, 60000) == 0
        tickets = []
        for i in subset:
            st, seed = reqs[i]
            t = ctypes.c_uint64()
            assert L.bingo_server_submit_walk(h, st.ctypes.data, len(st), ctypes.byref(pol), seed, ctypes.byref(t)) == 0
            tickets.append((i, t.value))
        out = {}
        for i, t in tickets:
            n = len(reqs[i][0])
            p = np.zeros((n, 41), np.uint32)
            l = np.zeros(n, np.uint32)
            ep = ctypes.c_uint64()
            assert L.bingo_server_wait(h, t, 60000, p.ctypes.data, l.ctypes.data, ctypes.byref(ep)) == 0
            out[i] = (p, l, ep.value)
        stats = B.bingo_server_stats()
        L.bingo_server_stats_get(h, ctypes.byref(stats))
        L.bingo_server_destroy(h)
        return out, stats

    mix, stats = serve(range(len(reqs)))
    assert stats.requests_done == len(reqs) and stats.p99_ms >= stats.p50_ms > 0
    for i in range(len(reqs)):
        alone, _ = serve([i])
        assert (alone[i][0] == mix[i][0]).all() and (alone[i][1] == mix[i][1]).all(), i
    # the same request equals a direct bingo_walk with its seed
    st, seed = reqs[2]
    p, l = run_walk(B, g, st, [pol], seed, 41)
    assert (p == mix[2][0]).all() and (l == mix[2][1]).all()
    # updates submitted to the server are applied at an epoch boundary before later requests
    og = O.Graph(G.n, G.row_ptr, G.col, G.w)
    upd = wl.batches[0].records()
    og.apply(upd, G.max_bits)
    after, stats2 = serve([3], updates=upd)
    assert after[3][2] >= 1 and stats2.updates_applied == len(upd)
    assert_steps_live(og, after[3][0], after[3][1])


def test_radix_base4_one_step_and_team_width(B):
    """Radix base 4: group 4^i then value sub-group v (weight v 4^i |S_iv|), then a uniform member;
    one-step frequencies match w / sum w, and every team width draws the same paths."""
    wl = W.make_workload("c2", scale=14, m=1 << 18, nbatch=1, batch=1000)
    G = wl.graph
    w = np.minimum(G.w, (1 << 20) - 1).astype(np.uint32)
    g = B.Graph(G.n, dev(G.row_ptr), dev(G.col), dev(w), max_bits=20, radix_base=4)
    og = O.Graph(G.n, G.row_ptr, G.col, w)
    assert og.set_base4() == 0
    offs, _, _, _ = og.edges()
    deg = np.diff(offs.astype(np.int64))
    for i, v in enumerate(np.argsort(-deg)[[0, 5, 50, 500]]):
        one_step_check(B, g, og, int(v), 600 + i)
    starts = W.walk_starts(G.n, 20000, 3)
    out = []
    for lanes in (1, 4, 32):
        g.set_walk_config(lanes, 8)
        out.append(run_walk(B, g, starts, [B.policy(B.DEEPWALK, 20)], 9, 21))
    for p, l in out[1:]:
        assert (p == out[0][0]).all() and (l == out[0][1]).all()
    assert_steps_live(og, *out[0])
