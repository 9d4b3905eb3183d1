"""Real-valued biases (Section 4.3) on the CUDA path, through the C ABI, against the oracle.

State parity is bit-exact: per edge the integer part I = floor(lambda b) and the
decimal part q = floor(frac(lambda b) 2^8); per vertex the radix groups of the
integer parts (counts, kinds, memberships) and the decimal total Q_D in group
slot 31.  Walks: one-step frequencies against (2^8 I + q) / sum at 10^6 samples
(TV <= 0.01, chi-square p > 1e-3), including decimal-only vertices and vertices
whose decimal parts are so small that the decimal group's rejection sampler
hands over to its inverse-transform fallback.
"""
import numpy as np
import pytest

import oracle as O
from tests.gpu_helpers import _segments, assert_steps_live, check_layout_invariants, gpu_canonical
from tests.stats import binned, chisq_p, tv

pytestmark = pytest.mark.gpu
N_SAMPLES = 1_000_000
LAM = 10.0


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


def f32bits(x):
    """binary32 encodings: an array for an array, an int for a scalar."""
    if np.ndim(x) == 0:
        return int(np.float32(x).view(np.uint32))
    return np.ascontiguousarray(np.asarray(x, dtype=np.float32)).view(np.uint32)


def real_biases(rng, size):
    """Mostly [0.5, 100) like the paper's float range; 10% below 1/lambda (decimal-only edges)."""
    b = rng.uniform(0.5, 100.0, size=size)
    small = rng.random(size) < 0.1
    b[small] = rng.uniform(0.02, 0.99, size=int(small.sum())) / LAM
    return b.astype(np.float32)


def real_graph(seed, n=96, hubs=6, hub_deg=120, base_deg=6, decimal_only=(7, 8)):
    """Multigraph covering every kind of integer group, with vertices whose biases are all below
    1/lambda (only the decimal group) and isolated vertices."""
    rng = np.random.default_rng(seed)
    edges = []
    for v in range(n):
        d = hub_deg if v < hubs else (0 if v % 11 == 5 else base_deg + int(rng.integers(0, 8)))
        bs = real_biases(rng, d)
        if v < hubs:  # mostly small biases, a few large: sparse and one-element high groups
            bs = np.where(rng.random(d) < 0.85, rng.uniform(0.05, 0.8, size=d), bs).astype(np.float32)
        if v in decimal_only:
            bs = (rng.uniform(0.02, 0.99, size=d) / LAM).astype(np.float32)
        for b in bs:
            edges.append((v, int(rng.integers(0, n)), f32bits(b)))
    og = O.Graph.from_edges(n, edges)
    assert og.set_lambda(LAM) == 0
    return og


def make(B, og):
    offs, dst, w, _ = og.edges()
    return B.Graph(og.n, dev(offs.astype(np.uint64)), dev(dst), dev(w), bias_format=B.BIAS_F32, lambda_=LAM)


def assert_real_state_matches(g, og, alpha=40, beta=10):
    ex = g.export_state()
    q = g.export_decimal()
    (gv, gd, gI, ge), (Gv, Gk, Ge) = gpu_canonical(ex)
    deg = ex["deg"].astype(np.int64)
    vslot = np.repeat(np.arange(len(deg), dtype=np.int64), deg)
    gq = q[np.lexsort((ex["eid"].astype(np.uint64), vslot))]
    offs, od, _, oe = og.edges()
    oI, oq, oqs = og.real_parts()
    ov = np.repeat(np.arange(og.n, dtype=np.int64), np.diff(offs.astype(np.int64)))
    assert len(ge) == len(oe), "edge count differs"
    assert (gv == ov).all() and (gd == od).all() and (ge == oe).all(), "adjacency differs"
    assert (gI == oI).all(), "integer parts differ"
    assert (gq.astype(np.uint32) == oq).all(), "decimal parts differ"
    cnt, kd, _ = og.factor_all(alpha, beta)
    assert (ex["cnt"][:, :31] == cnt[:, :31]).all(), "integer group counts differ"
    assert (ex["cnt"][:, 31].astype(np.uint64) == oqs).all(), "decimal totals differ"
    assert (ex["kind"] == kd).all() and (ex["kind"][:, 31] == O.EMPTY).all(), "group kinds differ"
    moffs, meids = og.members_all()
    glen = np.diff(moffs.astype(np.int64))
    Ov = np.repeat(np.arange(og.n * 32, dtype=np.int64) // 32, glen)
    Ok = np.repeat(np.arange(og.n * 32, dtype=np.int64) % 32, glen)
    assert len(Ge) == len(meids) and (Gv == Ov).all() and (Gk == Ok).all() and (Ge == meids).all(), \
        "group memberships differ"
    check_layout_invariants(ex)
    return ex


def real_batch(rng, og, n, size, hubs=6):
    offs, dst, _, _ = og.edges()
    rec = []
    for _ in range(size):
        op = rng.random()
        v = int(rng.integers(0, n)) if rng.random() < 0.6 else int(rng.integers(0, hubs))
        if op < 0.45:
            rec.append([v, int(rng.integers(0, n)), f32bits(real_biases(rng, 1)[0]), 0])
        elif op < 0.9:
            a, c = int(offs[v]), int(offs[v + 1])
            x = int(dst[int(rng.integers(a, c))]) if c > a and rng.random() < 0.9 else int(rng.integers(0, n))
            rec.append([v, x, 0, 1])
        else:
            a, c = int(offs[v]), int(offs[v + 1])
            x = int(dst[int(rng.integers(a, c))]) if c > a else int(rng.integers(0, n))
            rec.append([v, x, f32bits(real_biases(rng, 1)[0]), 2])
    return np.array(rec, dtype=np.uint32)


def apply_both(g, og, rec, stream=False):
    rec = np.ascontiguousarray(rec, dtype=np.uint32).reshape(-1, 4)
    if stream:
        st = g.stream_updates(dev(rec))
        tot = [0, 0, 0]
        for r in rec:
            rc, s = og.apply(r[None, :])
            assert rc == 0
            tot = [a + b for a, b in zip(tot, s)]
        ost = tuple(tot)
    else:
        st = g.apply_updates(dev(rec))
        rc, ost = og.apply(rec)
        assert rc == 0
    assert (st["inserted"], st["deleted"], st["not_found"]) == ost, (st, ost)
    return st


def test_real_create_matches_oracle(B):
    og = real_graph(1)
    g = make(B, og)
    ex = assert_real_state_matches(g, og)
    assert (ex["cnt"][7, :31] == 0).all() and ex["cnt"][7, 31] > 0, "decimal-only vertex"
    kinds = set(np.unique(ex["kind"]).tolist())
    assert {O.DENSE, O.ONE, O.SPARSE, O.REGULAR} <= kinds


@pytest.mark.parametrize("seed", [2, 3])
def test_real_batches_match_oracle(B, seed):
    og = real_graph(seed)
    g = make(B, og)
    rng = np.random.default_rng(50 + seed)
    for it in range(15):
        apply_both(g, og, real_batch(rng, og, og.n, [1, 5, 40, 200, 600][it % 5]))
        assert_real_state_matches(g, og)


def test_real_streaming_matches_oracle(B):
    og = real_graph(4)
    g = make(B, og)
    rng = np.random.default_rng(60)
    for it in range(3):
        apply_both(g, og, real_batch(rng, og, og.n, 150), stream=True)
        assert_real_state_matches(g, og)


def test_real_capacity_growth_moves_decimal_parts(B):
    n = 2048
    edges = [(0, 1 + j, f32bits(0.37 + j)) for j in range(3)] + [(1, 2 + j, f32bits(0.05)) for j in range(20)]
    og = O.Graph.from_edges(n, edges)
    assert og.set_lambda(LAM) == 0
    g = make(B, og)
    rng = np.random.default_rng(5)
    ins = np.array([[0, int(rng.integers(0, n)), f32bits(real_biases(rng, 1)[0]), 0] for _ in range(3000)],
                   np.uint32)
    apply_both(g, og, ins)
    assert_real_state_matches(g, og)
    apply_both(g, og, np.array([[1, 2 + j, 0, 1] for j in range(20)], np.uint32))
    ex = assert_real_state_matches(g, og)
    assert ex["deg"][1] == 0 and ex["cnt"][1, 31] == 0
    apply_both(g, og, np.array([[1, 9, f32bits(0.031), 0], [5, 9, f32bits(2.5), 0]], np.uint32))
    assert_real_state_matches(g, og)


def test_real_invalid_biases_rejected(B):
    og = real_graph(6)
    offs, dst, w, _ = og.edges()
    for bad in (np.nan, np.inf, -1.0, 0.0, 1e-6, 3e8):
        ww = w.copy()
        ww[5] = f32bits(bad)
        with pytest.raises(B.BingoError):
            B.Graph(og.n, dev(offs.astype(np.uint64)), dev(dst), dev(ww), bias_format=B.BIAS_F32, lambda_=LAM)
    g = make(B, og)
    before = g.export_decimal().copy()
    for bad in (np.nan, -2.0, 1e-6):
        with pytest.raises(B.BingoError):
            g.apply_updates(dev(np.array([[3, 4, f32bits(0.5), 0], [3, 5, f32bits(bad), 0]], np.uint32)))
    assert (g.export_decimal() == before).all()
    assert_real_state_matches(g, og)


def one_step_real(B, g, og, v, seed, n_samples=N_SAMPLES):
    offs, dst, _, _ = og.edges()
    I, q, _ = og.real_parts()
    a, c = int(offs[v]), int(offs[v + 1])
    d = dst[a:c].astype(np.int64)
    ww = I[a:c].astype(np.float64) * 256 + q[a:c]
    uniq, inv = np.unique(d, return_inverse=True)
    probs = np.bincount(inv, weights=ww)
    import torch

    paths = torch.empty((n_samples, 2), dtype=torch.int32, device="cuda")
    plen = torch.empty(n_samples, dtype=torch.int32, device="cuda")
    g.walk(dev(np.full(n_samples, v, np.uint32)), [B.policy(B.DEEPWALK, 1)], seed, 2, paths, plen)
    g.check()
    got = paths.cpu().numpy().view(np.uint32)[:, 1].astype(np.int64)
    assert (plen.cpu().numpy() == 2).all()
    pos = np.searchsorted(uniq, got)
    assert (uniq[np.minimum(pos, len(uniq) - 1)] == got).all(), "sampled a non-neighbour"
    counts = np.bincount(pos, minlength=len(uniq)).astype(np.float64)
    cb, pb = binned(counts, probs, 1000)
    tb, tpb = binned(counts, probs, 256)
    t, p = tv(tb, tpb), chisq_p(cb, pb)
    assert t <= 0.01 and p > 1e-3, (v, t, p)


def test_real_one_step_distribution(B):
    og = real_graph(8)
    g = make(B, og)
    for i, v in enumerate((0, 7, 8, 20, 41)):  # hubs, decimal-only vertices, plain vertices
        one_step_real(B, g, og, v, 310 + i)
    # the decimal group's sampler alone, with 32x the samples (power to see a 0.1% bias in a bin)
    one_step_real(B, g, og, 8, 320, n_samples=1 << 25)
    rng = np.random.default_rng(70)
    rec = real_batch(rng, og, og.n, 300)
    g.apply_updates(dev(rec))
    og.apply(rec)
    for i, v in enumerate((1, 7, 30)):
        one_step_real(B, g, og, v, 400 + i)


def test_real_decimal_fallback_is_exact(B):
    """Decimal parts of 1/256 on most edges: a candidate is accepted with probability ~1/256, so most
    draws from the decimal group end in the inverse-transform fallback; the law stays q / Q_D."""
    n = 64
    small = float(np.float32(1.5 / 256 / LAM))  # q = 1
    bs = [small] * 40 + [float(np.float32(0.09 / LAM))] * 3 + [float(np.float32(0.6 / LAM))]
    og = O.Graph.from_edges(n, [(0, 1 + j, f32bits(b)) for j, b in enumerate(bs)])
    assert og.set_lambda(LAM) == 0
    I, q, qs = og.real_parts()
    assert (I == 0).all() and q[0] == 1
    g = make(B, og)
    assert_real_state_matches(g, og)
    one_step_real(B, g, og, 0, 500)


def test_real_walks_live_and_team_independent(B):
    og = real_graph(9)
    g = make(B, og)
    rng = np.random.default_rng(80)
    starts = rng.integers(0, og.n, size=20000).astype(np.uint32)
    out = []
    for lanes in (1, 4, 32):
        g.set_walk_config(lanes, 8)
        import torch

        paths = torch.empty((len(starts), 41), dtype=torch.int32, device="cuda")
        plen = torch.empty(len(starts), dtype=torch.int32, device="cuda")
        g.walk(dev(starts), [B.policy(B.DEEPWALK, 40)], 7, 41, paths, plen)
        g.check()
        out.append((paths.cpu().numpy().view(np.uint32), plen.cpu().numpy().view(np.uint32)))
    for p, l in out[1:]:
        assert (p == out[0][0]).all() and (l == out[0][1]).all()
    assert_steps_live(og, *out[0])


def test_real_server_matches_direct_walk(B):
    """The serving loop on a real-bias graph: a request's paths equal a direct walk with its seed,
    alone or merged with others; real-bias updates go through the server's epochs."""
    import ctypes

    og = real_graph(10)
    g = make(B, og)
    L = B.load()
    pol = B.policy(B.DEEPWALK, 12)
    rng = np.random.default_rng(90)
    reqs = [(rng.integers(0, og.n, size=k).astype(np.uint32), 70 + i) for i, k in enumerate([3, 200, 1500])]
    h = ctypes.c_void_p()
    cfg = B.bingo_server_config()
    assert L.bingo_server_create(g.h, ctypes.byref(cfg), ctypes.byref(h)) == 0
    tickets = []
    for st, seed in reqs:
        t = ctypes.c_uint64()
        assert L.bingo_server_submit_walk(h, st.ctypes.data, len(st), ctypes.byref(pol), seed, ctypes.byref(t)) == 0
        tickets.append(t.value)
    out = []
    for (st, _), t in zip(reqs, tickets):
        p = np.zeros((len(st), 13), np.uint32)
        l = np.zeros(len(st), np.uint32)
        ep = ctypes.c_uint64()
        assert L.bingo_server_wait(h, t, 60000, p.ctypes.data, l.ctypes.data, ctypes.byref(ep)) == 0
        out.append((p, l))
    upd = real_batch(rng, og, og.n, 100)
    ep = ctypes.c_uint64()
    assert L.bingo_server_submit_updates(h, upd.ctypes.data, len(upd), ctypes.byref(ep)) == 0
    assert L.bingo_server_drain(h, 60000) == 0
    L.bingo_server_destroy(h)
    import torch

    for (st, seed), (p, l) in zip(reqs, out):
        paths = torch.empty((len(st), 13), dtype=torch.int32, device="cuda")
        plen = torch.empty(len(st), dtype=torch.int32, device="cuda")
        # the updates were applied after these requests: compare against a fresh graph of the old state
        g0 = make(B, real_graph(10))
        g0.walk(dev(st), [pol], seed, 13, paths, plen)
        g0.check()
        assert (paths.cpu().numpy().view(np.uint32) == p).all() and (plen.cpu().numpy().view(np.uint32) == l).all()
    og.apply(upd)
    assert_real_state_matches(g, og)
