"""Degenerate and extreme inputs on the CUDA path, against the oracle.

Graphs without edges, a single vertex with self-loops, the widest biases (all 32
bits, bit 31 alone: 64-bit totals and draws), the widest real biases (the
largest binary32 below 2^31) and the widest base-4 biases (every digit 3), each through
creation, updates and walks.
"""
import numpy as np
import pytest

import oracle as O
from tests.gpu_helpers import assert_state_matches, assert_steps_live
from tests.stats import binned, chisq_p, tv

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


def walk(B, g, starts, length, seed=1):
    import torch

    n = len(starts)
    paths = torch.empty((n, length + 1), dtype=torch.int32, device="cuda")
    plen = torch.empty(n, dtype=torch.int32, device="cuda")
    g.walk(dev(np.asarray(starts, dtype=np.uint32)), [B.policy(B.DEEPWALK, length)], seed, length + 1, paths, plen)
    g.check()
    return paths.cpu().numpy().view(np.uint32), plen.cpu().numpy().view(np.uint32)


def one_step(B, g, v, probs_by_dst, seed, n=1_000_000):
    paths, plen = walk(B, g, np.full(n, v), 1, seed)
    assert (plen == 2).all()
    uniq = np.array(sorted(probs_by_dst))
    pos = np.searchsorted(uniq, paths[:, 1].astype(np.int64))
    assert (uniq[np.minimum(pos, len(uniq) - 1)] == paths[:, 1]).all()
    counts = np.bincount(pos, minlength=len(uniq)).astype(np.float64)
    p = np.array([probs_by_dst[d] for d in uniq], dtype=np.float64)
    cb, pb = binned(counts, p, 1000)
    tb, tpb = binned(counts, p, 256)
    assert tv(tb, tpb) <= 0.01 and chisq_p(cb, pb) > 1e-3


def probs_of(edges, v, weight=lambda w: w):
    out = {}
    for s, d, w in edges:
        if s == v:
            out[d] = out.get(d, 0) + weight(w)
    tot = sum(out.values())
    return {d: x / tot for d, x in out.items()}


def test_graph_without_edges_then_filled_and_emptied(B):
    n = 16
    rp = np.zeros(n + 1, dtype=np.uint64)
    g = B.Graph(n, dev(rp), np.zeros(0, np.uint32), np.zeros(0, np.uint32))  # m = 0
    og = O.Graph(n, rp, np.zeros(0, np.uint32), np.zeros(0, np.uint32))
    ex = g.export_state()
    assert ex["deg"].sum() == 0 and (ex["kind"] == O.EMPTY).all()
    paths, plen = walk(B, g, np.arange(n), 5)
    assert (plen == 1).all() and (paths[:, 0] == np.arange(n)).all() and (paths[:, 1:] == 0xFFFFFFFF).all()
    rec = np.array([[v, (v + 1) % n, 1 + v, 0] for v in range(n)] + [[3, 4, 9, 0], [3, 4, 0, 1]], dtype=np.uint32)
    st = g.apply_updates(dev(rec))
    rc, ost = og.apply(rec)
    assert rc == 0 and (st["inserted"], st["deleted"], st["not_found"]) == ost
    assert_state_matches(g.export_state(), og)
    dels = np.array([[v, (v + 1) % n, 0, 1] for v in range(n)], dtype=np.uint32)
    g.apply_updates(dev(dels))
    og.apply(dels)
    ex = g.export_state()
    assert ex["deg"].sum() == 0
    assert_state_matches(ex, og)


def test_single_vertex_self_loops(B):
    edges = [(0, 0, 1), (0, 0, 6), (0, 0, 1 << 20)]
    og = O.Graph.from_edges(1, edges)
    offs, dst, w, _ = og.edges()
    g = B.Graph(1, dev(offs.astype(np.uint64)), dev(dst), dev(w))
    assert_state_matches(g.export_state(), og)
    paths, plen = walk(B, g, [0] * 100, 50)
    assert (plen == 51).all() and (paths == 0).all()


def test_widest_integer_biases(B):
    """Biases with all 32 bits set and bit 31 alone: group 31 and totals past 2^32 (64-bit draws)."""
    edges = [(0, 1, 0xFFFFFFFF), (0, 2, 1 << 31), (0, 3, 1), (0, 4, 3), (0, 5, 0x80000001)]
    edges += [(1, 0, 0xFFFFFFFF)] * 3 + [(1, 2, 7)]
    og = O.Graph.from_edges(6, edges)
    offs, dst, w, _ = og.edges()
    g = B.Graph(6, dev(offs.astype(np.uint64)), dev(dst), dev(w), max_bits=32)
    ex = g.export_state()
    assert_state_matches(ex, og)
    assert ex["cnt"][0, 31] == 3
    one_step(B, g, 0, probs_of(edges, 0), 11)
    one_step(B, g, 1, probs_of(edges, 1), 12)
    rec = np.array([[0, 3, 0xFFFFFFFE, 2], [1, 0, 0, 1], [2, 5, 1 << 31, 0]], dtype=np.uint32)
    g.apply_updates(dev(rec))
    og.apply(rec)
    assert_state_matches(g.export_state(), og)


def test_widest_real_biases(B):
    """Real biases at the largest binary32 below 2^31 (integer part 2^31 - 128, groups 7-30) beside
    pure decimal parts: totals in units of 2^-8 past 2^40."""
    lam = 1.0
    b = np.array([2147483520.0, 0.75, 3.5, 2147483520.0], dtype=np.float32)  # largest binary32 below 2^31
    bits = [int(x) for x in b.view(np.uint32)]
    edges = [(0, 1 + j, bits[j]) for j in range(4)]
    og = O.Graph.from_edges(8, edges)
    assert og.set_lambda(lam) == 0
    I, q, _ = og.real_parts()
    assert int(I[0]) == 2147483520 and int(q[1]) == 192
    offs, dst, w, _ = og.edges()
    g = B.Graph(8, dev(offs.astype(np.uint64)), dev(dst), dev(w), bias_format=B.BIAS_F32, lambda_=lam)
    ex = g.export_state()
    assert (g.export_decimal() == q.astype(np.uint8)).all()
    assert int(ex["cnt"][0, 31]) == int(q.sum())
    wts = {1 + j: int(I[j]) * 256 + int(q[j]) for j in range(4)}
    tot = sum(wts.values())
    paths, plen = walk(B, g, [0] * 200000, 1, 5)
    got = paths[:, 1]
    assert set(np.unique(got).tolist()) <= set(wts)
    # the two heavy edges take all but ~1e-9 of the mass
    assert ((got == 1) | (got == 4)).mean() > 0.999
    assert abs((got == 1).mean() - wts[1] / tot) < 0.01


def test_widest_base4_biases(B):
    """Every base-4 digit 3 (2^20 - 1): ten sub-groups of value 3, plus mixed digits."""
    edges = [(0, 1, (1 << 20) - 1), (0, 2, 0x55555), (0, 3, 0xAAAAA), (0, 4, 1), (0, 5, 2), (0, 6, 3)]
    og = O.Graph.from_edges(8, edges)
    assert og.set_base4() == 0
    offs, dst, w, _ = og.edges()
    g = B.Graph(8, dev(offs.astype(np.uint64)), dev(dst), dev(w), max_bits=20, radix_base=4)
    ex = g.export_state()
    assert_state_matches(ex, og, base4=True)
    assert (ex["bias"][:6] == w[:6]).all()
    one_step(B, g, 0, probs_of(edges, 0), 21)


def test_calls_with_nothing_to_do(B):
    """Zero walkers, an empty update batch and an empty streaming call are valid no-ops through every
    walk entry point and both buffer kinds, and leave the state exactly as created."""
    import torch

    edges = [(0, 1, 3), (1, 2, 5), (2, 0, 7), (2, 1, 1)]
    og = O.Graph.from_edges(3, edges)
    offs, dst, w, _ = og.edges()
    g = B.Graph(3, dev(offs.astype(np.uint64)), dev(dst), dev(w))
    pol = [B.policy(B.DEEPWALK, 4)]
    none_dev = torch.empty((0, 5), dtype=torch.int32, device="cuda")
    g.walk(torch.empty(0, dtype=torch.int32, device="cuda"), pol, 0, 5, none_dev,
           torch.empty(0, dtype=torch.int32, device="cuda"))
    g.walk(np.zeros(0, np.uint32), pol, 0, 5, np.zeros((0, 5), np.uint32), np.zeros(0, np.uint32))
    g.walk(np.zeros(0, np.uint32), pol, 0, 5, np.zeros((0, 5), np.uint32), np.zeros(0, np.uint32),
           mode=B.WALK_STEPWISE)
    g.check()
    st = g.apply_updates(torch.empty((0, 4), dtype=torch.int32, device="cuda"))
    assert (st["inserted"], st["deleted"], st["not_found"]) == (0, 0, 0)
    st = g.stream_updates(np.zeros((0, 4), np.uint32))
    assert (st["inserted"], st["deleted"], st["not_found"]) == (0, 0, 0)
    assert_state_matches(g.export_state(), og)
