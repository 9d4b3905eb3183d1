"""Seeded synthetic workloads: graphs, biases, update streams and walk starts.

This module only produces inputs.  The oracle tests and the CUDA path's tests
and bench both read their inputs from here, so both sides see identical bytes;
nothing here computes any step of the sampling method.

The five workloads mirror the paper's evaluation setup (Section 5.1: |V|
walkers, length 80, batches of updates between walks, power-law graphs) with
synthetic RMAT / Erdos-Renyi graphs standing in for the paper's datasets, which
are not available here.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_LIB = os.path.join(_HERE, "libbingo_workloads.so")
_lock = threading.Lock()
_lib = None

U32P = ctypes.POINTER(ctypes.c_uint32)
U64P = ctypes.POINTER(ctypes.c_uint64)
U8P = ctypes.POINTER(ctypes.c_uint8)


def build(force: bool = False) -> str:
    """Compile gen.c into a shared library next to it (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _L():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            c = ctypes
            sig = {
                "wl_philox4x32_10": (None, [U32P, U32P, U32P]),
                "wl_walk_starts": (None, [c.c_uint32, c.c_uint64, c.c_uint64, U32P]),
                "wl_er": (None, [c.c_uint32, c.c_uint64, c.c_uint64, U32P, U32P]),
                "wl_relabel": (c.c_uint32, [c.c_uint32, c.c_uint32, c.c_uint64]),
                "wl_rmat": (None, [c.c_uint32, c.c_uint64, c.c_double, c.c_double, c.c_double, c.c_uint64, U32P, U32P]),
                "wl_hubs": (None, [c.c_uint32, c.c_uint32, c.c_uint64, c.c_uint64, U32P, U32P, U32P]),
                "wl_bias_uniform": (None, [c.c_uint64, c.c_uint32, c.c_uint32, c.c_uint64, U32P]),
                "wl_bias_pareto15": (None, [c.c_uint64, c.c_uint32, c.c_uint64, U32P]),
                "wl_bias_fixed": (None, [c.c_uint64, c.c_uint32, c.c_uint32, c.c_uint64, U32P]),
                "wl_to_csr": (None, [c.c_uint32, c.c_uint64, U32P, U32P, U32P, U64P, U32P, U32P]),
                "wl_update_stream": (c.c_int, [c.c_uint64, U32P, U32P, U32P, c.c_uint32, c.c_uint64, c.c_uint64,
                                               c.c_uint64, U8P, U32P, U32P, U32P, U32P]),
                "wl_uniform_batch": (None, [c.c_uint32, c.c_uint64, U64P, U32P, c.c_uint64, c.c_uint64, c.c_uint32,
                                            c.c_uint32, c.c_uint64, U32P, U32P, U32P, U32P]),
                "wl_shuffle_updates": (None, [c.c_uint64, c.c_uint64, U32P, U32P, U32P, U32P]),
                "wl_uniform01": (None, [c.c_uint64, c.c_uint64, c.c_uint64, ctypes.POINTER(c.c_double)]),
            }
            for name, (res, args) in sig.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    t = {np.uint32: U32P, np.uint64: U64P, np.uint8: U8P, np.float64: ctypes.POINTER(ctypes.c_double)}[a.dtype.type]
    return a.ctypes.data_as(t)


# ---------------------------------------------------------------------------------------------
# primitives


def philox4x32_10(ctr, key) -> np.ndarray:
    """Philox4x32-10 (Salmon et al., SC'11) on one counter; used for input draws only."""
    c = np.asarray(ctr, dtype=np.uint32).copy()
    k = np.asarray(key, dtype=np.uint32).copy()
    o = np.zeros(4, dtype=np.uint32)
    _L().wl_philox4x32_10(_p(c), _p(k), _p(o))
    return o


def walk_starts(n: int, count: int, seed: int = 0) -> np.ndarray:
    """Uniform start vertices: start_i = floor(philox(i,0,0,0; seed).x * n / 2^32)."""
    out = np.empty(count, dtype=np.uint32)
    _L().wl_walk_starts(n, count, seed, _p(out))
    return out


def er_edges(n: int, m: int, seed: int):
    s = np.empty(m, dtype=np.uint32)
    d = np.empty(m, dtype=np.uint32)
    _L().wl_er(n, m, seed, _p(s), _p(d))
    return s, d


def rmat_edges(scale: int, m: int, seed: int, a=0.57, b=0.19, c=0.19):
    s = np.empty(m, dtype=np.uint32)
    d = np.empty(m, dtype=np.uint32)
    _L().wl_rmat(scale, m, a, b, c, seed, _p(s), _p(d))
    return s, d


def hub_edges(n: int, nhubs: int, per_hub: int, seed: int):
    ids = np.empty(nhubs, dtype=np.uint32)
    s = np.empty(nhubs * per_hub, dtype=np.uint32)
    d = np.empty(nhubs * per_hub, dtype=np.uint32)
    _L().wl_hubs(n, nhubs, per_hub, seed, _p(ids), _p(s), _p(d))
    return ids, s, d


def biases(m: int, spec, seed: int) -> np.ndarray:
    """spec: ("uniform", lo, hi_excl) | ("pareto15", cap) | ("fixed", lo, hi_excl)."""
    w = np.empty(m, dtype=np.uint32)
    kind = spec[0]
    if kind == "uniform":
        _L().wl_bias_uniform(m, spec[1], spec[2], seed, _p(w))
    elif kind == "pareto15":
        _L().wl_bias_pareto15(m, spec[1], seed, _p(w))
    elif kind == "fixed":
        _L().wl_bias_fixed(m, spec[1], spec[2], seed, _p(w))
    else:
        raise ValueError(spec)
    return w


def to_csr(n: int, src: np.ndarray, dst: np.ndarray, w: np.ndarray):
    """Stable counting sort by source -> (row_ptr u64[n+1], col u32[m], w u32[m])."""
    m = len(src)
    rp = np.empty(n + 1, dtype=np.uint64)
    col = np.empty(m, dtype=np.uint32)
    wo = np.empty(m, dtype=np.uint32)
    _L().wl_to_csr(n, m, _p(np.ascontiguousarray(src)), _p(np.ascontiguousarray(dst)),
                   _p(np.ascontiguousarray(w)), _p(rp), _p(col), _p(wo))
    return rp, col, wo


def uniform01(count: int, seed: int, stream: int = 0) -> np.ndarray:
    out = np.empty(count, dtype=np.float64)
    _L().wl_uniform01(count, seed, stream, _p(out))
    return out


# ---------------------------------------------------------------------------------------------
# update records


@dataclasses.dataclass
class Updates:
    src: np.ndarray
    dst: np.ndarray
    bias: np.ndarray
    op: np.ndarray  # 0 insert, 1 delete, 2 set_bias

    def __len__(self):
        return len(self.src)

    def slice(self, a: int, b: int) -> "Updates":
        return Updates(self.src[a:b], self.dst[a:b], self.bias[a:b], self.op[a:b])

    def records(self) -> np.ndarray:
        """Packed array of 16-byte records {src, dst, bias, op} (the C-ABI's bingo_update)."""
        r = np.empty((len(self), 4), dtype=np.uint32)
        r[:, 0], r[:, 1], r[:, 2], r[:, 3] = self.src, self.dst, self.bias, self.op
        return r


def uniform_batch(n, row_ptr, col, nins, ndel, wlo, whi, seed, shuffle=True) -> Updates:
    m = int(row_ptr[-1])
    cnt = nins + ndel
    s, d, w, o = (np.empty(cnt, dtype=np.uint32) for _ in range(4))
    _L().wl_uniform_batch(n, m, _p(np.ascontiguousarray(row_ptr, dtype=np.uint64)),
                          _p(np.ascontiguousarray(col, dtype=np.uint32)), nins, ndel, wlo, whi, seed,
                          _p(s), _p(d), _p(w), _p(o))
    if shuffle:
        _L().wl_shuffle_updates(cnt, seed, _p(s), _p(d), _p(w), _p(o))
    return Updates(s, d, w, o)


# ---------------------------------------------------------------------------------------------
# the five workloads


@dataclasses.dataclass
class Graph:
    n: int
    row_ptr: np.ndarray
    col: np.ndarray
    w: np.ndarray
    max_bits: int

    @property
    def m(self) -> int:
        return int(self.row_ptr[-1])


@dataclasses.dataclass
class Workload:
    name: str
    graph: Graph
    batches: list  # list[Updates]
    nwalkers: int
    length: int
    walk_seed: int
    extra: dict


CONFIGS = {
    # ER directed 1,024 / 16,384, biases U[1,255]; 1,024 walkers x 80; one batch of 1,024 + 1,024.
    "c1": dict(graph="er", n=1024, m=16384, bias=("uniform", 1, 256), max_bits=8, graph_seed=1,
               nwalkers=1024, length=80, walk_seed=0, updates=("uniform", 1, 1024, 1024)),
    # RMAT-20, Pareto(1.5) biases clipped to 2^20; 1M DeepWalk x 80; 10 batches of 10^5 (50/50).
    "c2": dict(graph="rmat", scale=20, m=1 << 24, bias=("pareto15", 1 << 20), max_bits=21, graph_seed=2,
               nwalkers=1 << 20, length=80, walk_seed=0, updates=("stream", 10, 50000, 50000)),
    # RMAT-24, fixed-point biases w_fx in [128, 25600) (w = w_fx / 256); 4M mixed node2vec + PPR.
    "c3": dict(graph="rmat", scale=24, m=1 << 28, bias=("fixed", 128, 25600), max_bits=15, graph_seed=3,
               nwalkers=4 << 20, length=80, walk_seed=0, updates=None),
    # RMAT-22, U[1, 2^16); serving with a Poisson update stream (70% insert).
    "c4": dict(graph="rmat", scale=22, m=1 << 26, bias=("uniform", 1, 1 << 16), max_bits=16, graph_seed=4,
               nwalkers=10000, length=40, walk_seed=5, updates=("stream", 10, 70000, 30000)),
    # RMAT-26 + 64 hubs of 10^6 extra edges, U[1, 2^31); batch sweep between rounds of 16M PPR.
    "c5": dict(graph="rmat", scale=26, m=1 << 30, hubs=(64, 10 ** 6), bias=("uniform", 1, 1 << 31), max_bits=31,
               graph_seed=6, nwalkers=16 << 20, length=100, walk_seed=0, updates=("stream", 5, 5_000_000, 5_000_000)),
}


def make_workload(name: str, scale: int | None = None, m: int | None = None, nbatch: int | None = None,
                  batch: int | None = None, nwalkers: int | None = None, hubs: bool = True) -> Workload:
    """Build a workload.  `scale`/`m`/`nbatch`/`batch`/`nwalkers` shrink it for tests; hubs=False leaves
    out a recipe's hub edges (profiling cases of the plain RMAT part).

    For the "stream" update protocol the graph generator produces m + (#inserts)
    edges; the held-out ones become the inserts (Section 5.1, datasets), so the
    initial graph has exactly m edges.
    """
    cfg = CONFIGS[name]
    gseed = cfg["graph_seed"]
    if cfg["graph"] == "er":
        n = cfg["n"] if scale is None else (1 << scale)
        mm = cfg["m"] if m is None else m
    else:
        sc = cfg["scale"] if scale is None else scale
        n = 1 << sc
        mm = cfg["m"] if m is None else m
    upd = cfg["updates"]
    nb = ins = dele = 0
    if upd is not None and upd[0] == "stream":
        nb = upd[1] if nbatch is None else nbatch
        tot = upd[2] + upd[3]
        if batch is not None:
            frac = upd[2] / tot
            ins = int(round(batch * frac))
            dele = batch - ins
        else:
            ins, dele = upd[2], upd[3]
    n_extra = nb * ins
    total = mm + n_extra
    if cfg["graph"] == "er":
        s, d = er_edges(n, total, gseed)
    else:
        s, d = rmat_edges(int(np.log2(n)), total, gseed)
    want_hubs = hubs
    hubs = None
    if "hubs" in cfg and want_hubs:
        nh, per = cfg["hubs"]
        if scale is not None:
            per = max(1, min(per, mm // 16))
        hubs, hs, hd = hub_edges(n, nh, per, gseed + 1000)
        s = np.concatenate([s, hs])
        d = np.concatenate([d, hd])
    w = biases(len(s), cfg["bias"], gseed)
    batches = []
    if upd is not None and upd[0] == "stream":
        keep = np.empty(len(s), dtype=np.uint8)
        cnt = nb * (ins + dele)
        us, ud, uw, uo = (np.empty(cnt, dtype=np.uint32) for _ in range(4))
        rc = _L().wl_update_stream(len(s), _p(s), _p(d), _p(w), nb, ins, dele, gseed + 77, _p(keep),
                                   _p(us), _p(ud), _p(uw), _p(uo))
        if rc != 0:
            raise RuntimeError(f"update stream generation failed ({rc})")
        k = keep.astype(bool)
        s, d, w = s[k], d[k], w[k]
        per = ins + dele
        allu = Updates(us, ud, uw, uo)
        batches = [allu.slice(i * per, (i + 1) * per) for i in range(nb)]
    rp, col, wc = to_csr(n, s, d, w)
    g = Graph(n=n, row_ptr=rp, col=col, w=wc, max_bits=cfg["max_bits"])
    if upd is not None and upd[0] == "uniform":
        nb = upd[1] if nbatch is None else nbatch
        ni, nd = upd[2], upd[3]
        if batch is not None:
            ni, nd = batch // 2, batch - batch // 2
        lo, hi = (cfg["bias"][1], cfg["bias"][2]) if cfg["bias"][0] != "pareto15" else (1, 256)
        batches = [uniform_batch(n, rp, col, ni, nd, lo, hi, gseed + 101 + i) for i in range(nb)]
    nw = cfg["nwalkers"] if nwalkers is None else nwalkers
    return Workload(name=name, graph=g, batches=batches, nwalkers=nw, length=cfg["length"],
                    walk_seed=cfg["walk_seed"], extra={"hubs": hubs})
