"""bingo_walk_packed: the same walks as bingo_walk, each path without its padding, packed in walker order."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def _t(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_packed_equals_padded_rows_device_and_host():
    import torch

    import paper_2504_10233_gb300 as B

    wl = W.make_workload("c2", scale=14, m=1 << 18, nbatch=1, batch=2000)
    G = wl.graph
    g = B.Graph(G.n, _t(G.row_ptr), _t(G.col), _t(G.w), max_bits=G.max_bits)
    nw, L = 40000, 50
    starts_h = W.walk_starts(G.n, nw, 4)
    pids_h = (np.arange(nw) % 3).astype(np.uint8)
    pols = [B.policy(B.DEEPWALK, L), B.policy(B.PPR, L, 0.15), B.policy(B.NODE2VEC, L - 7, n2v_pq=(2.0, 0.5))]
    ref_p = torch.empty((nw, L + 1), dtype=torch.int32, device="cuda")
    ref_l = torch.empty(nw, dtype=torch.int32, device="cuda")
    g.walk(_t(starts_h), pols, 31, L + 1, ref_p, ref_l, policy_ids=_t(pids_h))
    g.check()
    rp, rl = ref_p.cpu().numpy().view(np.uint32), ref_l.cpu().numpy().view(np.uint32)
    exp = np.concatenate([rp[i, :rl[i]] for i in range(nw)])
    # device buffers
    dl = torch.zeros(nw, dtype=torch.int32, device="cuda")
    dv = torch.full((nw * (L + 1),), -1, dtype=torch.int32, device="cuda")
    tot = g.walk_packed(_t(starts_h), pols, 31, L, dl, dv, policy_ids=_t(pids_h))
    assert tot == int(rl.astype(np.int64).sum()) == len(exp)
    assert (dl.cpu().numpy().view(np.uint32) == rl).all()
    assert (dv[:tot].cpu().numpy().view(np.uint32) == exp).all()
    assert (dv[tot:].cpu().numpy() == -1).all(), "entries past the total are not written"
    # host buffers (pageable numpy and pinned torch)
    for make in (lambda n: np.zeros(n, np.uint32), lambda n: torch.zeros(n, dtype=torch.int32).pin_memory()):
        hl, hv = make(nw), make(nw * (L + 1))
        tot = g.walk_packed(starts_h, pols, 31, L, hl, hv, policy_ids=pids_h)
        hl_np = hl if isinstance(hl, np.ndarray) else hl.numpy().view(np.uint32)
        hv_np = hv if isinstance(hv, np.ndarray) else hv.numpy().view(np.uint32)
        assert (hl_np == rl).all() and (hv_np[:tot] == exp).all()
    # per-walker lengths: the same as bingo_walk with those lengths
    lens = (np.arange(nw) * 7 % (L + 1)).astype(np.uint32)
    g.walk(_t(starts_h), pols, 32, L + 1, ref_p, ref_l, lengths=_t(lens), policy_ids=_t(pids_h))
    rp, rl = ref_p.cpu().numpy().view(np.uint32), ref_l.cpu().numpy().view(np.uint32)
    exp = np.concatenate([rp[i, :rl[i]] for i in range(nw)])
    tot = g.walk_packed(_t(starts_h), pols, 32, L, dl, dv, lengths=_t(lens), policy_ids=_t(pids_h))
    assert tot == len(exp) and (dv[:tot].cpu().numpy().view(np.uint32) == exp).all()
    # too small a capacity: lengths and the total are reported, the vertices are not written
    small = np.full(10, 7, np.uint32)
    with pytest.raises(B.BingoError) as e:
        g.walk_packed(starts_h, pols, 31, L, np.zeros(nw, np.uint32), small, policy_ids=pids_h)
    assert e.value.status == B.E_INVALID and (small == 7).all()
    # a step limit above max_steps is reported
    with pytest.raises(B.BingoError):
        g.walk_packed(_t(starts_h), pols, 31, L - 1, dl, dv, policy_ids=_t(pids_h))
    g.check()
    g.close()
