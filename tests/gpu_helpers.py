"""Comparison of the CUDA path's exported state with the oracle, and walk checks.

The GPU export is brought to the oracle's canonical form (edges by vertex and
edge id; every group (v, k) as an ascending set of edge ids) and compared
element by element.  Layout (member positions, inverted indexes, sparse
lists) has no oracle counterpart and is checked here by its invariants.
"""
from __future__ import annotations

import numpy as np

import oracle as O

KINDS = (O.EMPTY, O.DENSE, O.ONE, O.SPARSE, O.REGULAR)


def _segments(lengths):
    lengths = np.asarray(lengths, dtype=np.int64)
    starts = np.zeros(len(lengths), dtype=np.int64)
    if len(lengths) > 1:
        starts[1:] = np.cumsum(lengths)[:-1]
    return starts


def b4_slots(w):
    """Radix base 4: slot mask of each bias (bit 3 i + v - 1 for every nonzero base-4 digit v at
    position i), from the digits of the base-4 numeral."""
    out = np.zeros(len(w), dtype=np.uint64)
    for j, x in enumerate(np.asarray(w, dtype=np.int64)):
        for i, ch in enumerate(reversed(np.base_repr(int(x), 4))):
            if ch != "0":
                out[j] |= np.uint64(1) << np.uint64(3 * i + int(ch) - 1)
    return out


def gpu_canonical(ex, memb=None, skip_dense=False):
    """Edges sorted by (vertex, eid) and group memberships sorted by (vertex, k, eid).  memb: per
    edge slot mask when it is not the bias itself (radix base 4).  skip_dense: leave out dense groups,
    whose members are by definition the adjacency filtered by bit k (compared through the adjacency
    and the kinds)."""
    deg = ex["deg"].astype(np.int64)
    n = len(deg)
    eoff = _segments(deg)
    vslot = np.repeat(np.arange(n, dtype=np.int64), deg)
    eid = ex["eid"].astype(np.uint64)
    order = np.lexsort((eid, vslot))
    edges = (vslot[order], ex["dst"][order], ex["bias"][order], eid[order])
    # groups: (v, k, eid) for every membership
    kind = ex["kind"]
    w = (ex["bias"] if memb is None else memb).astype(np.uint64)
    vs, ks, es = [], [], []
    # dense groups: filter the adjacency by bit k
    for k in (range(32) if not skip_dense else ()):
        bit = ((w >> np.uint64(k)) & np.uint64(1)).astype(bool)
        dense_v = kind[:, k] == O.DENSE
        sel = bit & dense_v[vslot]
        vs.append(vslot[sel]); ks.append(np.full(int(sel.sum()), k, np.int64)); es.append(eid[sel])
    # one-element groups
    ov, ok = np.nonzero(kind == O.ONE)
    oslot = ex["one_slot"][ov, ok].astype(np.int64)
    vs.append(ov.astype(np.int64)); ks.append(ok.astype(np.int64)); es.append(eid[eoff[ov] + oslot])
    # list groups
    glen = ex["glen"].reshape(-1).astype(np.int64)
    gv = np.repeat(np.arange(n * 32, dtype=np.int64) // 32, glen)
    gk = np.repeat(np.arange(n * 32, dtype=np.int64) % 32, glen)
    mem = ex["members"].astype(np.int64)
    gkind = kind[gv, gk]
    sp_off = _segments(ex["sp_len"])
    slot = mem.copy()
    sp = gkind == O.SPARSE
    slot[sp] = ex["sp_list"][sp_off[gv[sp]] + mem[sp]].astype(np.int64)
    vs.append(gv); ks.append(gk); es.append(eid[eoff[gv] + slot])
    V, K, E = np.concatenate(vs), np.concatenate(ks), np.concatenate(es)
    o = np.lexsort((E, K, V))
    return edges, (V[o], K[o], E[o])


def oracle_canonical(og: O.Graph):
    offs, dst, w, eid = og.edges()
    deg = np.diff(offs.astype(np.int64))
    v = np.repeat(np.arange(og.n, dtype=np.int64), deg)
    moffs, meids = og.members_all()
    glen = np.diff(moffs.astype(np.int64))
    gv = np.repeat(np.arange(og.n * 32, dtype=np.int64) // 32, glen)
    gk = np.repeat(np.arange(og.n * 32, dtype=np.int64) % 32, glen)
    return (v, dst, w, eid), (gv, gk, meids.astype(np.uint64))


def check_layout_invariants(ex, memb=None):
    """Member lists compact and consistent with their inverted indexes; sparse lists exact."""
    wbits = (ex["bias"] if memb is None else memb).astype(np.uint64)
    deg = ex["deg"].astype(np.int64)
    n = len(deg)
    kind = ex["kind"]
    cnt = ex["cnt"].astype(np.int64)
    glen = ex["glen"].astype(np.int64)
    listk = (kind == O.REGULAR) | (kind == O.SPARSE)
    assert (glen[listk] == cnt[listk]).all(), "list length != |G_k|"
    assert (glen[~listk] == 0).all()
    gl = glen.reshape(-1)
    pos = np.arange(gl.sum(), dtype=np.int64) - np.repeat(_segments(gl), gl)
    assert (ex["member_inv"].astype(np.int64) == pos).all(), "inverted index does not point back at its member"
    gv = np.repeat(np.arange(n * 32, dtype=np.int64) // 32, gl)
    gk = np.repeat(np.arange(n * 32, dtype=np.int64) % 32, gl)
    mem = ex["members"].astype(np.int64)
    reg = kind[gv, gk] == O.REGULAR
    assert (mem[reg] < deg[gv[reg]]).all(), "regular member outside the adjacency"
    spl = ex["sp_len"].astype(np.int64)
    sp = ~reg
    assert (mem[sp] < spl[gv[sp]]).all(), "sparse member outside the sparse list"
    # members distinct within each group
    key = gv * 32 + gk
    pairs = np.unique(np.stack([key, mem]), axis=1)
    assert pairs.shape[1] == len(mem), "duplicate member in a group"
    # sparse list: inverse consistent, entries = edges in any sparse group
    spos = np.arange(spl.sum(), dtype=np.int64) - np.repeat(_segments(spl), spl)
    assert (ex["sp_inv"].astype(np.int64) == spos).all(), "sparse-list inverted index inconsistent"
    spmask = np.zeros(n, dtype=np.uint64)
    sv, sk = np.nonzero(kind == O.SPARSE)
    np.bitwise_or.at(spmask, sv, (np.uint64(1) << sk.astype(np.uint64)))
    eoff = _segments(deg)
    vslot = np.repeat(np.arange(n, dtype=np.int64), deg)
    in_s = (wbits & spmask[vslot]) != 0
    exp_cnt = np.bincount(vslot[in_s], minlength=n)
    assert (exp_cnt == spl).all(), "sparse list size != edges in sparse groups"
    sv2 = np.repeat(np.arange(n, dtype=np.int64), spl)
    slots = ex["sp_list"].astype(np.int64)
    assert (slots < deg[sv2]).all()
    assert in_s[eoff[sv2] + slots].all(), "sparse list holds an edge of no sparse group"
    # one-element slots hold the bit
    ov, ok = np.nonzero(kind == O.ONE)
    os_ = ex["one_slot"][ov, ok].astype(np.int64)
    assert (os_ < deg[ov]).all()
    assert (((wbits[eoff[ov] + os_] >> ok.astype(np.uint64)) & np.uint64(1)) == 1).all()


def assert_state_matches(ex, og: O.Graph, alpha=40, beta=10, base4=False):
    """Bit-exact factorisation state (edges, |G_k|, kinds, memberships) + layout invariants."""
    memb = b4_slots(ex["bias"]) if base4 else None
    (gv, gd, gw, ge), (Gv, Gk, Ge) = gpu_canonical(ex, memb)
    (ov, od, ow, oe), (Ov, Ok, Oe) = oracle_canonical(og)
    assert len(ge) == len(oe), f"edge count {len(ge)} != oracle {len(oe)}"
    assert (gv == ov).all() and (gd == od).all() and (gw == ow).all() and (ge == oe).all(), "adjacency differs"
    cnt, kd, sw = og.factor_all(alpha, beta)
    assert (ex["cnt"] == cnt).all(), "group counts differ"
    assert (ex["kind"] == kd).all(), "group kinds differ"
    assert len(Ge) == len(Oe), f"membership count {len(Ge)} != oracle {len(Oe)}"
    assert (Gv == Ov).all() and (Gk == Ok).all() and (Ge == Oe).all(), "group memberships differ"
    check_layout_invariants(ex, memb)


def edge_keys(og: O.Graph):
    offs, dst, _, _ = og.edges()
    deg = np.diff(offs.astype(np.int64))
    src = np.repeat(np.arange(og.n, dtype=np.uint64), deg)
    return np.unique((src << np.uint64(32)) | dst.astype(np.uint64))


def assert_steps_live(og: O.Graph, paths: np.ndarray, plen: np.ndarray, keys=None, padded=True):
    """Every consecutive pair of every path is a live edge of the oracle graph; padding is 0xFFFFFFFF
    (padded=False: entries past path_len are the caller's and are not looked at)."""
    keys = edge_keys(og) if keys is None else keys
    L = paths.shape[1]
    idx = np.arange(L - 1)[None, :]
    valid = idx < (plen.astype(np.int64)[:, None] - 1)
    u = paths[:, :-1][valid].astype(np.uint64)
    x = paths[:, 1:][valid].astype(np.uint64)
    q = (u << np.uint64(32)) | x
    pos = np.searchsorted(keys, q)
    pos = np.minimum(pos, len(keys) - 1)
    ok = keys[pos] == q
    assert ok.all(), f"{int((~ok).sum())} steps are not live edges"
    if padded:
        pad = np.arange(L)[None, :] >= plen.astype(np.int64)[:, None]
        assert (paths[pad] == 0xFFFFFFFF).all(), "padding is not 0xFFFFFFFF"


def assert_vertices_match(exv, og: O.Graph, ids, alpha=40, beta=10):
    """Bit-exact state of listed vertices (bingo_export_vertices rows) against an oracle graph holding
    at least those vertices' rows: adjacency (destination, bias, edge id), |G_k| and kinds, and the
    member sets of every one-element, sparse and regular group; layout invariants of the rows.  Dense
    groups are the adjacency filtered by bit k on both sides, so the adjacency and kind comparisons
    cover them."""
    ids = np.asarray(ids, dtype=np.uint32)
    k = len(ids)
    (gv, gd, gw, ge), (Gv, Gk, Ge) = gpu_canonical(exv, skip_dense=True)
    offs, od, ow, oe = og.edges_of(ids)
    odeg = np.diff(offs.astype(np.int64))
    ov = np.repeat(np.arange(k, dtype=np.int64), odeg)
    assert (exv["deg"].astype(np.int64) == odeg).all(), "degrees differ"
    assert len(ge) == len(oe), f"edge count {len(ge)} != oracle {len(oe)}"
    assert (gv == ov).all() and (gd == od).all() and (gw == ow).all() and (ge == oe).all(), "adjacency differs"
    cnt = np.zeros((k, 32), dtype=np.uint32)
    kd = np.zeros((k, 32), dtype=np.uint8)
    for i, v in enumerate(ids):
        cnt[i], kd[i], _ = og.factor(int(v), alpha, beta)
    assert (exv["cnt"] == cnt).all(), "group counts differ"
    assert (exv["kind"] == kd).all(), "group kinds differ"
    # members of the non-dense groups by definition: the edges whose bias has bit k (Eq. dwi)
    vs, ks, es = [], [], []
    listlike = (kd == O.ONE) | (kd == O.SPARSE) | (kd == O.REGULAR)
    keep = listlike.any(axis=1)[ov]  # only rows with a non-dense group have members to compare
    ov_, w64, oe_ = ov[keep], ow[keep].astype(np.uint64), oe[keep]
    for b in range(32):
        sel = (((w64 >> np.uint64(b)) & np.uint64(1)) == 1) & listlike[ov_, b]
        vs.append(ov_[sel]); ks.append(np.full(int(sel.sum()), b, np.int64)); es.append(oe_[sel])
    V, K, E = np.concatenate(vs), np.concatenate(ks), np.concatenate(es).astype(np.uint64)
    o = np.lexsort((E, K, V))
    assert len(Ge) == len(E), f"membership count {len(Ge)} != oracle {len(E)}"
    assert (Gv == V[o]).all() and (Gk == K[o]).all() and (Ge == E[o]).all(), "group memberships differ"
    check_layout_invariants(exv)


def sampled_oracle(G, ids, next_eid=None):
    """Oracle graph holding only the rows of the listed sources of CSR graph G, each edge with its id
    in G (its CSR position); other vertices have no edges."""
    ids = np.unique(np.asarray(ids, dtype=np.int64))
    rp = G.row_ptr.astype(np.int64)
    deg = rp[ids + 1] - rp[ids]
    sub_rp = np.zeros(G.n + 1, dtype=np.int64)
    sub_rp[ids + 1] = deg
    sub_rp = np.cumsum(sub_rp).astype(np.uint64)
    tot = int(deg.sum())
    rows = np.repeat(rp[ids], deg) + (np.arange(tot, dtype=np.int64) - np.repeat(np.cumsum(deg) - deg, deg))
    return O.Graph.from_csr_ids(G.n, sub_rp, G.col[rows], G.w[rows], rows.astype(np.uint64),
                                int(rp[-1]) if next_eid is None else next_eid)


def insertion_ids(records, next_eid):
    """Edge id of every insertion record of a batch: the count continues in batch order (Section 5.2)."""
    op = np.asarray(records)[:, 3]
    ins = (op == 0) | (op == 2)
    return (next_eid + np.cumsum(ins) - 1).astype(np.uint64), next_eid + int(ins.sum())
