"""bingo_walk_noalloc: the walk for callers that cannot allocate device memory.

Callers inside allocator or memory-pool callbacks, under frameworks that have
reserved all device memory, or in loops that forbid cudaMalloc/cudaFree use
this entry point; it must return exactly what bingo_walk returns (paths are
integer vertex ids, so the comparison is exact) while allocating nothing.
This file is collected last so that a failure here never hides another test.
"""
import ctypes
import os
import subprocess
import sys

import numpy as np
import pytest

import workloads as W
from tests.conftest import ROOT

pytestmark = pytest.mark.gpu


def _dev(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_noalloc_walk_matches_bingo_walk_on_two_calls():
    import torch

    assert torch.cuda.is_available(), "GPU test"
    from paper_2504_10233_gb300 import _build

    _build.build()
    import paper_2504_10233_gb300 as B

    L = B.load()
    wl = W.make_workload("c2", scale=14, m=1 << 18, nbatch=1, batch=2000)
    G = wl.graph
    g = B.Graph(G.n, _dev(G.row_ptr), _dev(G.col), _dev(G.w), max_bits=G.max_bits)
    nw, stride = 30000, 41
    starts = _dev(W.walk_starts(G.n, nw, 3))
    pids = _dev((np.arange(nw) % 3).astype(np.uint8))
    pols = [B.policy(B.DEEPWALK, 40), B.policy(B.PPR, 40, 0.15), B.policy(B.NODE2VEC, 40, n2v_pq=(2.0, 0.5))]
    arr = (B.bingo_policy * 3)(*pols)

    def out():
        return (torch.full((nw, stride), -7, dtype=torch.int32, device="cuda"),
                torch.zeros(nw, dtype=torch.int32, device="cuda"))

    for call, seed in enumerate((11, 12)):  # two calls in a row share the fixed scratch
        ref_p, ref_l = out()
        B.bingo_walk(g.h, nw, starts, pols, seed, stride, ref_p, ref_l, policy_ids=pids)  # also builds the edge index
        g.check()
        p, l = out()
        st = L.bingo_walk_noalloc(g.h, nw, starts.data_ptr(), None, pids.data_ptr(), arr, 3, seed, stride,
                                  p.data_ptr(), l.data_ptr(), B.WALK_PERSISTENT, None)
        assert st == B.OK, L.bingo_last_error()
        g.check()
        assert torch.equal(p, ref_p) and torch.equal(l, ref_l), f"call {call}: differs from bingo_walk"

    # limits: more policies than the fixed table holds, host buffers, the stepwise form
    many = (B.bingo_policy * 17)(*([pols[0]] * 17))
    p, l = out()
    assert L.bingo_walk_noalloc(g.h, nw, starts.data_ptr(), None, None, many, 17, 1, stride, p.data_ptr(),
                                l.data_ptr(), 0, None) == B.E_INVALID
    host_starts = np.zeros(4, np.uint32)
    assert L.bingo_walk_noalloc(g.h, 4, host_starts.ctypes.data, None, None, arr, 1, 1, stride, p.data_ptr(),
                                l.data_ptr(), 0, None) == B.E_INVALID
    assert L.bingo_walk_noalloc(g.h, nw, starts.data_ptr(), None, None, arr, 1, 1, stride, p.data_ptr(),
                                l.data_ptr(), B.WALK_STEPWISE, None) == B.E_INVALID
    g.close()


def test_noalloc_node2vec_needs_an_edge_index_and_lengths_path():
    """node2vec on a graph whose edge index was never built (only bingo_walk builds it, and building
    allocates) is refused with BINGO_E_STATE; per-walker lengths give what bingo_walk gives."""
    import torch

    import paper_2504_10233_gb300 as B

    L = B.load()
    wl = W.make_workload("c1")
    G = wl.graph
    g = B.Graph(G.n, _dev(G.row_ptr), _dev(G.col), _dev(G.w), max_bits=G.max_bits)
    nw, stride = 2048, 81
    starts = _dev(W.walk_starts(G.n, nw, 5))
    p = torch.zeros((nw, stride), dtype=torch.int32, device="cuda")
    l = torch.zeros(nw, dtype=torch.int32, device="cuda")
    n2v = (B.bingo_policy * 1)(B.policy(B.NODE2VEC, 80, n2v_pq=(2.0, 0.5)))
    assert L.bingo_walk_noalloc(g.h, nw, starts.data_ptr(), None, None, n2v, 1, 3, stride, p.data_ptr(),
                                l.data_ptr(), 0, None) == B.E_STATE
    lengths = _dev((np.arange(nw) * 7919 % 81).astype(np.uint32))  # 0..80 steps, zero-length walkers included
    pol = (B.bingo_policy * 1)(B.policy(B.DEEPWALK, 80))
    ref_p, ref_l = torch.full_like(p, -3), torch.zeros_like(l)
    B.bingo_walk(g.h, nw, starts, [pol[0]], 21, stride, ref_p, ref_l, lengths=lengths)
    g.check()
    for _ in range(2):
        p.fill_(-5)
        assert L.bingo_walk_noalloc(g.h, nw, starts.data_ptr(), lengths.data_ptr(), None, pol, 1, 21, stride,
                                    p.data_ptr(), l.data_ptr(), 0, None) == B.OK, L.bingo_last_error()
        g.check()
        assert torch.equal(p, ref_p) and torch.equal(l, ref_l)
    g.close()


_FRESH = r"""
import sys
sys.path.insert(0, sys.argv[1])
import numpy as np, torch
import paper_2504_10233_gb300 as B, workloads as W
L = B.load()
wl = W.make_workload("c2", scale=14, m=1 << 18, nbatch=1, batch=2000)
G = wl.graph
t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
g = B.Graph(G.n, t(G.row_ptr), t(G.col), t(G.w), max_bits=G.max_bits)
nw, stride = 50000, 41
starts = t(W.walk_starts(G.n, nw, 3))
pids = t((np.arange(nw) % 2).astype(np.uint8))
pol = (B.bingo_policy * 2)(B.policy(B.DEEPWALK, 40), B.policy(B.PPR, 40, 0.15))
p = torch.zeros((nw, stride), dtype=torch.int32, device="cuda")
l = torch.zeros(nw, dtype=torch.int32, device="cuda")
torch.cuda.synchronize()
free0 = torch.cuda.mem_get_info()[0]
for seed in (1, 2):  # the first walk of any kind in this process, then a second one
    st = L.bingo_walk_noalloc(g.h, nw, starts.data_ptr(), None, pids.data_ptr(), pol, 2, seed, stride, p.data_ptr(),
                              l.data_ptr(), 0, None)
    assert st == 0, L.bingo_last_error()
    torch.cuda.synchronize()
free1 = torch.cuda.mem_get_info()[0]
g.check()
assert int(l.min()) >= 1
print("FREE", free0, free1)
"""


def test_noalloc_first_call_in_a_fresh_process_allocates_nothing():
    """In a process that has created a graph but never walked, the first two no-alloc walks leave the
    device's free memory unchanged: bingo_create loaded the walker kernels and resolved the scratch
    array, so the call neither loads a module nor allocates."""
    from paper_2504_10233_gb300 import _build

    _build.build()
    r = subprocess.run([sys.executable, "-c", _FRESH, ROOT], capture_output=True, text=True, timeout=600,
                       env=dict(os.environ, PYTHONPATH=ROOT))
    assert r.returncode == 0, r.stdout + r.stderr
    line = [x for x in r.stdout.splitlines() if x.startswith("FREE ")][-1]
    free0, free1 = (int(x) for x in line.split()[1:])
    assert free1 == free0, f"device free memory changed by {free0 - free1} bytes across the first no-alloc calls"
