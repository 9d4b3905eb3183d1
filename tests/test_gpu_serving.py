"""Admission in the serving loop, tested with host-side means only.

A request is admitted while the walker slots in flight plus its own stay within
max_inflight_walkers and its launch buffers leave hbm_reserve_bytes of device memory free;
otherwise it waits in the queue.  Each case holds a request back on purpose (admission paused,
slots taken by an earlier request, free memory below the reserve until the test frees some),
checks that bingo_server_wait times out with the request still queued or that it was admitted
only after the earlier request completed, and that once admitted its paths equal a direct
bingo_walk with its seed.
"""
import ctypes
import time

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch

    assert torch.cuda.is_available(), "GPU test"
    import paper_2504_10233_gb300 as B

    L = B.load()
    wl = W.make_workload("c4", scale=14, m=1 << 18, nbatch=1, batch=1000)
    G = wl.graph
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    g = B.Graph(G.n, t(G.row_ptr), t(G.col), t(G.w), max_bits=G.max_bits)
    yield B, L, G, g
    g.close()


def _server(B, L, g, **cfg_kw):
    cfg = B.bingo_server_config()
    for k, v in cfg_kw.items():
        setattr(cfg, k, v)
    h = ctypes.c_void_p()
    assert L.bingo_server_create(g.h, ctypes.byref(cfg), ctypes.byref(h)) == 0
    return h


def _submit(B, L, h, starts, pol, seed):
    tk = ctypes.c_uint64()
    assert L.bingo_server_submit_walk(h, starts.ctypes.data, len(starts), ctypes.byref(pol), seed, ctypes.byref(tk)) == 0
    return tk.value


def _info(B, L, h, tk):
    info = B.bingo_server_request_info()
    assert L.bingo_server_request_get(h, tk, ctypes.byref(info)) == 0
    return info


def _wait(B, L, h, tk, n, stride, timeout_ms=60000):
    p = np.zeros((n, stride), np.uint32)
    l = np.zeros(n, np.uint32)
    ep = ctypes.c_uint64()
    st = L.bingo_server_wait(h, tk, timeout_ms, p.ctypes.data, l.ctypes.data, ctypes.byref(ep))
    return st, p, l


def _direct(B, g, starts, pol, seed, stride):
    p = np.zeros((len(starts), stride), np.uint32)
    l = np.zeros(len(starts), np.uint32)
    g.walk(starts, [pol], seed, stride, p, l)
    return p, l


def _until_done(B, L, h, tickets, timeout_s=60):
    t_end = time.time() + timeout_s
    while time.time() < t_end:
        if all(_info(B, L, h, tk).state == 2 for tk in tickets):
            return
        time.sleep(0.002)
    raise AssertionError("requests did not complete")


def test_paused_request_stays_queued_then_completes(env):
    B, L, G, g = env
    pol = B.policy(B.PPR, 40, 0.15)
    h = _server(B, L, g)
    assert L.bingo_server_pause(h, 1) == 0
    st = W.walk_starts(G.n, 300, 1)
    tk = _submit(B, L, h, st, pol, 77)
    code, _, _ = _wait(B, L, h, tk, 300, 41, timeout_ms=150)
    assert code == B.E_TIMEOUT
    info = _info(B, L, h, tk)
    assert info.state == 0 and info.admit_ms < 0 and info.walkers == 300
    assert L.bingo_server_pause(h, 0) == 0
    code, p, l = _wait(B, L, h, tk, 300, 41)
    assert code == B.OK
    L.bingo_server_destroy(h)  # the server owns the graph until here
    rp, rl = _direct(B, g, st, pol, 77, 41)
    assert (p == rp).all() and (l == rl).all()


def test_request_waits_for_walker_slots(env):
    """Two requests queued together while admission is paused: A takes every walker slot, so B (which
    cannot join A's launch) is admitted only after A's launch has completed."""
    B, L, G, g = env
    pol = B.policy(B.DEEPWALK, 100)
    h = _server(B, L, g, max_inflight_walkers=4000, max_len_cap=128)
    assert L.bingo_server_pause(h, 1) == 0
    sa, sb = W.walk_starts(G.n, 4000, 2), W.walk_starts(G.n, 16, 3)
    ta, tb = _submit(B, L, h, sa, pol, 5), _submit(B, L, h, sb, pol, 6)
    assert L.bingo_server_pause(h, 0) == 0
    _until_done(B, L, h, [ta, tb])
    ia, ib = _info(B, L, h, ta), _info(B, L, h, tb)
    assert 0 <= ia.admit_ms <= ia.done_ms <= ib.admit_ms <= ib.done_ms, (ia.admit_ms, ia.done_ms, ib.admit_ms)
    got = []
    for tk, st, seed in ((ta, sa, 5), (tb, sb, 6)):
        code, p, l = _wait(B, L, h, tk, len(st), 101)
        assert code == B.OK
        got.append((st, seed, p, l))
    L.bingo_server_destroy(h)
    for st, seed, p, l in got:
        rp, rl = _direct(B, g, st, pol, seed, 101)
        assert (p == rp).all() and (l == rl).all()


def test_request_waits_for_free_device_memory(env):
    """The reserve is set above the free memory left while the test holds a buffer; the request stays
    queued until the buffer is released, then runs and equals a direct walk."""
    import torch

    B, L, G, g = env
    pol = B.policy(B.PPR, 40, 0.15)
    held = torch.empty(4 << 30, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    free_now = torch.cuda.mem_get_info()[0]
    h = _server(B, L, g, hbm_reserve_bytes=free_now + (2 << 30))
    st = W.walk_starts(G.n, 500, 4)
    tk = _submit(B, L, h, st, pol, 91)
    code, _, _ = _wait(B, L, h, tk, 500, 41, timeout_ms=300)
    assert code == B.E_TIMEOUT and _info(B, L, h, tk).state == 0
    del held
    torch.cuda.empty_cache()
    _until_done(B, L, h, [tk])
    info = _info(B, L, h, tk)
    assert info.admit_ms >= info.submit_ms + 300
    code, p, l = _wait(B, L, h, tk, 500, 41)
    assert code == B.OK
    L.bingo_server_destroy(h)
    rp, rl = _direct(B, g, st, pol, 91, 41)
    assert (p == rp).all() and (l == rl).all()
