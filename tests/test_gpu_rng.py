"""The walker's random numbers on the device, pinned to published values and other implementations.

Walks draw from Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) with counter (walker lo, walker
hi, step, j) and key (seed lo, seed hi), and turn words into exact uniform integers by Lemire's
multiply-shift with rejection (ACM TOMACS 2019).  Checked here, on the device code the walker runs:
the Random123 known-answer vectors (tests/golden/philox_kat.json); agreement with cuRAND's
curand_Philox4x32_10 and with the host implementation of the input generators on random counters
and keys; the per-step counter stream and the bounded draws word for word; and, end to end through
bingo_walk, PPR walk lengths equal to the ones the counter layout predicts exactly.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import workloads as W
from tests.conftest import ROOT, golden

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import torch

    assert torch.cuda.is_available(), "GPU test"
    import paper_2504_10233_gb300 as B

    B.load()
    return B


@pytest.fixture(scope="module")
def curand_lib(tmp_path_factory):
    src = os.path.join(ROOT, "tests", "native", "curand_philox.cu")
    out = str(tmp_path_factory.mktemp("curand") / "libcurand_philox_ref.so")
    subprocess.check_call(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-shared", "-Xcompiler",
                           "-fPIC", "-o", out, src])
    lib = ctypes.CDLL(out)
    lib.curand_philox_ref.restype = ctypes.c_int
    lib.curand_philox_ref.argtypes = [ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    return lib


def _host_philox(ctr, key):
    return np.stack([W.philox4x32_10(c, k) for c, k in zip(ctr, key)]).astype(np.uint32)


def test_device_philox_known_answer_vectors(B):
    vecs = golden("philox_kat.json")["vectors"]
    ctr = np.array([[int(x, 16) for x in v["ctr"]] for v in vecs], dtype=np.uint32)
    key = np.array([[int(x, 16) for x in v["key"]] for v in vecs], dtype=np.uint32)
    exp = np.array([[int(x, 16) for x in v["out"]] for v in vecs], dtype=np.uint32)
    assert np.array_equal(B.bingo_philox4x32_10(ctr, key), exp)


def test_device_philox_matches_curand_and_host(B, curand_lib):
    rng = np.random.default_rng(2024)
    n = 4096
    ctr = rng.integers(0, 1 << 32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 1 << 32, size=(n, 2), dtype=np.uint64).astype(np.uint32)
    ctr[:8] = 0  # small and extreme counters too
    ctr[8:16] = 0xFFFFFFFF
    dev = B.bingo_philox4x32_10(ctr, key)
    ref = np.zeros_like(ctr)
    assert curand_lib.curand_philox_ref(n, ctr.ctypes.data, key.ctypes.data, ref.ctypes.data) == 0
    assert np.array_equal(dev, ref), "device Philox differs from cuRAND's curand_Philox4x32_10"
    assert np.array_equal(dev[:512], _host_philox(ctr[:512], key[:512]))


CASES = [(0, 0, 0), (0, 1, 0), (7, 12345, 79), (0x0123456789ABCDEF, (1 << 32) + 5, 3), ((1 << 64) - 1, (1 << 40) - 1, 99)]


def _stream(seed, walker, step, nwords):
    key = [seed & 0xFFFFFFFF, seed >> 32]
    words = []
    j = 0
    while len(words) < nwords:
        words += [int(x) for x in W.philox4x32_10([walker & 0xFFFFFFFF, walker >> 32, step, j], key)]
        j += 1
    return words


def test_walker_counter_stream(B):
    for seed, walker, step in CASES:
        got = B.bingo_walker_draws(seed, walker, step, 12)
        assert [int(x) for x in got] == _stream(seed, walker, step, 12), (seed, walker, step)


def _lemire(words, rng_range, count):
    """Exact uniform integers in [0, range) from a word stream (Lemire 2019, with rejection)."""
    it = iter(words)
    out = []
    for _ in range(count):
        if rng_range < 1 << 32:
            m = next(it) * rng_range
            if m % (1 << 32) < rng_range:
                t = ((1 << 32) - rng_range) % rng_range
                while m % (1 << 32) < t:
                    m = next(it) * rng_range
            out.append(m >> 32)
        else:
            x = (next(it) << 32) | next(it)
            m = x * rng_range
            if m % (1 << 64) < rng_range:
                t = ((1 << 64) - rng_range) % rng_range
                while m % (1 << 64) < t:
                    x = (next(it) << 32) | next(it)
                    m = x * rng_range
            out.append(m >> 64)
    return out


def test_walker_bounded_draws(B):
    ranges = [1, 2, 3, 1000, (1 << 31) + 1, (1 << 32) - 1, 1 << 32, (1 << 32) + 5, (1 << 40) + 3, (1 << 63) + 7]
    for seed, walker, step in CASES[:3]:
        words = _stream(seed, walker, step, 2 * 64 * 3)
        for r in ranges:
            got = [int(x) for x in B.bingo_walker_draws(seed, walker, step, 64, r)]
            assert got == _lemire(words, r, 64), (r, seed, walker, step)
            assert all(0 <= x < r for x in got)


def test_ppr_lengths_follow_the_counter_layout(B):
    """On a graph where every vertex has an out-edge only the stop rule ends a PPR walk, and the stop
    test is the first word of each step's stream: walker i stops before step s iff
    philox((i lo, i hi, s, 0), key).x < ppr_stop_u32, so its length is known exactly."""
    import torch

    n = 256
    rp = np.arange(n + 1, dtype=np.uint64) * 2
    col = np.stack([(np.arange(n) + 1) % n, (np.arange(n) * 5 + 3) % n], axis=1).reshape(-1).astype(np.uint32)
    w = np.tile(np.array([3, 5], dtype=np.uint32), n)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    g = B.Graph(n, t(rp), t(col), t(w), max_bits=8)
    nw, cap, seed = 3000, 30, 0x5EED0000000A
    thr = B.policy(B.PPR, cap, 0.15).ppr_stop_u32
    starts = t(W.walk_starts(n, nw, 9))
    paths = torch.empty((nw, cap + 1), dtype=torch.int32, device="cuda")
    plen = torch.empty(nw, dtype=torch.int32, device="cuda")
    key = [seed & 0xFFFFFFFF, seed >> 32]
    exp = np.full(nw, cap)
    for i in range(nw):
        for s in range(cap):
            if int(W.philox4x32_10([i, 0, s, 0], key)[0]) < thr:
                exp[i] = s
                break
    assert 0 < (exp < cap).mean() < 1
    for lanes in (1, 4, 32):
        g.set_walk_config(lanes, 8)
        g.walk(starts, [B.policy(B.PPR, cap, 0.15)], seed, cap + 1, paths, plen)
        g.check()
        got = plen.cpu().numpy().astype(np.int64) - 1
        assert np.array_equal(got, exp), f"lanes {lanes}"
    g.close()
