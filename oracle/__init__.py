"""Python handle on the CPU oracle (oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by
the bench's CPU-baseline leg.  The product path never imports this package.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

EMPTY, DENSE, ONE, SPARSE, REGULAR = 0, 1, 2, 3, 4
KIND_NAMES = {EMPTY: "empty", DENSE: "dense", ONE: "one", SPARSE: "sparse", REGULAR: "regular"}
DEEPWALK, PPR, NODE2VEC = 0, 1, 2
PAD = 0xFFFFFFFF

c = ctypes
U32P = c.POINTER(c.c_uint32)
U64P = c.POINTER(c.c_uint64)
U8P = c.POINTER(c.c_uint8)
DP = c.POINTER(c.c_double)


class OPolicy(c.Structure):
    _fields_ = [("kind", c.c_uint32), ("max_len", c.c_uint32), ("ppr_stop_u32", c.c_uint32),
                ("pad", c.c_uint32), ("n2v_accept", c.c_uint64 * 3)]


def build(force: bool = False) -> str:
    """Compile oracle.c (gcc -O2, OpenMP) into liboracle.so next to it."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _L():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = c.CDLL(_LIB)
            sig = {
                "o_create": (c.c_void_p, [c.c_uint32, U64P, U32P, U32P]),
                "o_create_ids": (c.c_void_p, [c.c_uint32, U64P, U32P, U32P, U64P, c.c_uint64]),
                "o_apply_ids": (c.c_int, [c.c_void_p, U32P, c.c_uint64, c.c_uint32, U64P, U64P]),
                "o_edges_of": (None, [c.c_void_p, U32P, c.c_uint64, U64P, U32P, U32P, U64P]),
                "o_degree_sum": (c.c_uint64, [c.c_void_p, U32P, c.c_uint64]),
                "o_count_edges": (None, [c.c_void_p, U32P, U32P, c.c_uint64, U32P]),
                "o_destroy": (None, [c.c_void_p]),
                "o_num_edges": (c.c_uint64, [c.c_void_p]),
                "o_degree": (c.c_uint32, [c.c_void_p, c.c_uint32]),
                "o_export_edges": (None, [c.c_void_p, U64P, U32P, U32P, U64P]),
                "o_has_edge": (c.c_int, [c.c_void_p, c.c_uint32, c.c_uint32]),
                "o_apply": (c.c_int, [c.c_void_p, U32P, c.c_uint64, c.c_uint32, U64P]),
                "o_kind": (c.c_int, [c.c_uint64, c.c_uint64, c.c_uint32, c.c_uint32]),
                "o_factor": (None, [c.c_void_p, c.c_uint32, c.c_uint32, c.c_uint32, U32P, U8P, U64P]),
                "o_factor_all": (None, [c.c_void_p, c.c_uint32, c.c_uint32, U32P, U8P, U64P]),
                "o_group_totals": (None, [c.c_void_p, c.c_uint32, U64P]),
                "o_members_count": (c.c_uint64, [c.c_void_p]),
                "o_members_all": (None, [c.c_void_p, U64P, U64P]),
                "o_factored_prob": (c.c_int, [c.c_void_p, c.c_uint32, c.c_uint64, c.c_uint32, c.c_uint32, U64P, U64P]),
                "o_its_pick": (c.c_uint64, [c.c_void_p, c.c_uint32, c.c_uint64]),
                "o_n2v_weights": (None, [c.c_void_p, c.c_uint32, c.c_uint32, U64P, U64P]),
                "o_walk": (None, [c.c_void_p, c.c_uint64, U32P, U32P, U8P, c.POINTER(OPolicy), c.c_uint64,
                                  c.c_uint64, U32P, U32P]),
                "o_sample_many": (None, [c.c_void_p, c.c_uint32, c.c_uint64, c.c_uint64, U64P]),
                "o_num_threads": (c.c_int, []),
                "o_set_threads": (None, [c.c_int]),
                "o_float_factor": (None, [c.c_uint64, DP, c.c_double, U32P, U64P, DP, DP]),
                "o_set_lambda": (c.c_int, [c.c_void_p, c.c_double]),
                "o_set_base4": (c.c_int, [c.c_void_p]),
                "o_export_real": (None, [c.c_void_p, U32P, U32P, U64P]),
            }
            for name, (res, args) in sig.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def _p(a):
    assert a.flags["C_CONTIGUOUS"], "array must be contiguous"
    t = {np.uint32: U32P, np.uint64: U64P, np.uint8: U8P, np.float64: DP}[a.dtype.type]
    return a.ctypes.data_as(t)


ALL_REGULAR = 0xFFFFFFFF  # alpha value of the paper's BS baseline: every nonempty group regular


def kind(cnt: int, d: int, alpha: int = 40, beta: int = 10) -> int:
    return _L().o_kind(cnt, d, alpha, beta)


def num_threads() -> int:
    return _L().o_num_threads()


def set_threads(n: int) -> None:
    """Threads of the oracle's OpenMP loops from now on."""
    _L().o_set_threads(int(n))


def policy(kind_: int, max_len: int, ppr_stop_u32: int = 0, n2v_accept=(0, 0, 0)) -> OPolicy:
    p = OPolicy()
    p.kind, p.max_len, p.ppr_stop_u32, p.pad = kind_, max_len, ppr_stop_u32, 0
    for i in range(3):
        p.n2v_accept[i] = int(n2v_accept[i])
    return p


class Graph:
    """Oracle graph: explicit adjacency lists, edge ids 0..m-1 in CSR order."""

    def __init__(self, n: int, row_ptr, col, w):
        self.n = int(n)
        rp = np.ascontiguousarray(row_ptr, dtype=np.uint64)
        co = np.ascontiguousarray(col, dtype=np.uint32)
        ww = np.ascontiguousarray(w, dtype=np.uint32)
        self._h = _L().o_create(self.n, _p(rp), _p(co), _p(ww))
        if not self._h:
            raise MemoryError("oracle graph")

    @classmethod
    def from_csr_ids(cls, n: int, row_ptr, col, w, eid, next_eid: int):
        """Oracle graph from CSR rows whose edges carry explicit ids (ascending within each row); later
        insertions continue from next_eid.  Used to hold only some sources' rows of a larger graph."""
        self = cls.__new__(cls)
        self.n = int(n)
        rp = np.ascontiguousarray(row_ptr, dtype=np.uint64)
        co = np.ascontiguousarray(col, dtype=np.uint32)
        ww = np.ascontiguousarray(w, dtype=np.uint32)
        ee = np.ascontiguousarray(eid, dtype=np.uint64)
        self._h = _L().o_create_ids(self.n, _p(rp), _p(co), _p(ww), _p(ee), int(next_eid))
        if not self._h:
            raise MemoryError("oracle graph")
        return self

    @classmethod
    def from_edges(cls, n, edges):
        """edges: iterable of (src, dst, w) in edge-id order (stable by source)."""
        e = sorted(enumerate(edges), key=lambda t: (t[1][0], t[0]))
        rp = np.zeros(n + 1, dtype=np.uint64)
        for _, (s, _, _) in e:
            rp[s + 1] += 1
        rp = np.cumsum(rp).astype(np.uint64)
        col = np.array([x[1][1] for x in e], dtype=np.uint32)
        w = np.array([x[1][2] for x in e], dtype=np.uint32)
        return cls(n, rp, col, w)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            _L().o_destroy(h)
            self._h = None

    @property
    def m(self) -> int:
        return int(_L().o_num_edges(self._h))

    def degree(self, v: int) -> int:
        return int(_L().o_degree(self._h, v))

    def has_edge(self, u: int, x: int) -> bool:
        return bool(_L().o_has_edge(self._h, u, x))

    def apply(self, records: np.ndarray, max_bits: int = 32):
        """records: [count][4] u32 {src, dst, bias, op}. Returns (status, (inserted, deleted, not_found))."""
        r = np.ascontiguousarray(records, dtype=np.uint32).reshape(-1, 4)
        st = np.zeros(3, dtype=np.uint64)
        rc = _L().o_apply(self._h, _p(r), r.shape[0], max_bits, _p(st))
        return rc, tuple(int(x) for x in st)

    def apply_ids(self, records: np.ndarray, ins_ids, max_bits: int = 32):
        """apply() with the edge id of every insertion given (ins_ids[i] for record i; ignored for
        deletions).  Returns (status, (inserted, deleted, not_found))."""
        r = np.ascontiguousarray(records, dtype=np.uint32).reshape(-1, 4)
        ids = np.ascontiguousarray(ins_ids, dtype=np.uint64)
        assert len(ids) == r.shape[0]
        st = np.zeros(3, dtype=np.uint64)
        rc = _L().o_apply_ids(self._h, _p(r), r.shape[0], max_bits, _p(ids), _p(st))
        return rc, tuple(int(x) for x in st)

    def count_edges(self, us, xs):
        """Live copies of every (us[i], xs[i])."""
        us = np.ascontiguousarray(us, dtype=np.uint32)
        xs = np.ascontiguousarray(xs, dtype=np.uint32)
        out = np.zeros(len(us), dtype=np.uint32)
        _L().o_count_edges(self._h, _p(us), _p(xs), len(us), _p(out))
        return out

    def edges_of(self, ids):
        """(offs u64[k+1], dst, w, eid) of the listed vertices (row i = ids[i]), ascending eid."""
        ids = np.ascontiguousarray(ids, dtype=np.uint32)
        m = int(_L().o_degree_sum(self._h, _p(ids), len(ids)))
        offs = np.empty(len(ids) + 1, dtype=np.uint64)
        dst = np.empty(max(m, 1), dtype=np.uint32)
        w = np.empty(max(m, 1), dtype=np.uint32)
        eid = np.empty(max(m, 1), dtype=np.uint64)
        _L().o_edges_of(self._h, _p(ids), len(ids), _p(offs), _p(dst), _p(w), _p(eid))
        return offs, dst[:m], w[:m], eid[:m]

    def set_lambda(self, lam: float) -> int:
        """Real-valued biases (Section 4.3): stored words are binary32 encodings, weights
        2^8 floor(lam b) + floor(frac(lam b) 2^8).  Returns the status (0 = ok)."""
        return int(_L().o_set_lambda(self._h, float(lam)))

    def set_base4(self) -> int:
        """Radix base 4 (Appendix): sub-group (i, v) of digit position i and value v in slot
        3 i + v - 1, carrying v 4^i per member.  Returns the status (0 = ok)."""
        return int(_L().o_set_base4(self._h))

    def real_parts(self):
        """(I u32[m], q u32[m], qsum u64[n]): integer and decimal parts per edge in the order of
        edges(), and the decimal total per vertex."""
        m = self.m
        I = np.empty(m, dtype=np.uint32)
        q = np.empty(m, dtype=np.uint32)
        qs = np.empty(self.n, dtype=np.uint64)
        _L().o_export_real(self._h, _p(I), _p(q), _p(qs))
        return I, q, qs

    def edges(self):
        """(offs u64[n+1], dst u32[m], w u32[m], eid u64[m]) per vertex in ascending eid order."""
        m = self.m
        offs = np.empty(self.n + 1, dtype=np.uint64)
        dst = np.empty(m, dtype=np.uint32)
        w = np.empty(m, dtype=np.uint32)
        eid = np.empty(m, dtype=np.uint64)
        _L().o_export_edges(self._h, _p(offs), _p(dst), _p(w), _p(eid))
        return offs, dst, w, eid

    def factor(self, v: int, alpha=40, beta=10):
        cnt = np.zeros(32, dtype=np.uint32)
        kd = np.zeros(32, dtype=np.uint8)
        sw = np.zeros(1, dtype=np.uint64)
        _L().o_factor(self._h, v, alpha, beta, _p(cnt), _p(kd), _p(sw))
        return cnt, kd, int(sw[0])

    def factor_all(self, alpha=40, beta=10):
        cnt = np.zeros((self.n, 32), dtype=np.uint32)
        kd = np.zeros((self.n, 32), dtype=np.uint8)
        sw = np.zeros(self.n, dtype=np.uint64)
        _L().o_factor_all(self._h, alpha, beta, _p(cnt), _p(kd), _p(sw))
        return cnt, kd, sw

    def group_totals(self, v: int):
        W = np.zeros(32, dtype=np.uint64)
        _L().o_group_totals(self._h, v, _p(W))
        return W

    def members_all(self):
        """(offs u64[32n+1], eids u64[...]): ascending edge ids of every group (v, k)."""
        tot = int(_L().o_members_count(self._h))
        offs = np.empty(32 * self.n + 1, dtype=np.uint64)
        eids = np.empty(max(tot, 1), dtype=np.uint64)
        _L().o_members_all(self._h, _p(offs), _p(eids))
        return offs, eids[:tot]

    def factored_prob(self, v: int, i: int, alpha=40, beta=10):
        num = np.zeros(1, dtype=np.uint64)
        den = np.zeros(1, dtype=np.uint64)
        rc = _L().o_factored_prob(self._h, v, i, alpha, beta, _p(num), _p(den))
        if rc:
            raise ValueError("vertex has no edges")
        return int(num[0]), int(den[0])

    def its_pick(self, v: int, r: int) -> int:
        return int(_L().o_its_pick(self._h, v, r))

    def n2v_weights(self, prev: int, u: int, accept):
        a = np.ascontiguousarray(np.asarray(accept, dtype=np.uint64))
        out = np.zeros(max(self.degree(u), 1), dtype=np.uint64)
        _L().o_n2v_weights(self._h, prev, u, _p(a), _p(out))
        return out[: self.degree(u)]

    def walk(self, starts, policies, seed: int, lengths=None, policy_ids=None, stride=None):
        starts = np.ascontiguousarray(starts, dtype=np.uint32)
        nw = len(starts)
        pols = (OPolicy * len(policies))(*policies)
        maxlen = max(p.max_len for p in policies) if lengths is None else int(np.max(lengths, initial=0))
        stride = maxlen + 1 if stride is None else stride
        paths = np.empty((nw, stride), dtype=np.uint32)
        plen = np.empty(nw, dtype=np.uint32)
        lp = _p(np.ascontiguousarray(lengths, dtype=np.uint32)) if lengths is not None else None
        if policy_ids is not None:
            policy_ids = np.ascontiguousarray(policy_ids, dtype=np.uint8)
        pp = _p(policy_ids) if policy_ids is not None else None
        _L().o_walk(self._h, nw, _p(starts), lp, pp, pols, seed, stride, _p(paths), _p(plen))
        return paths, plen

    def sample_many(self, v: int, count: int, seed: int):
        out = np.empty(count, dtype=np.uint64)
        _L().o_sample_many(self._h, v, count, seed, _p(out))
        return out


def float_factor(biases, lam: float):
    b = np.ascontiguousarray(biases, dtype=np.float64)
    cnt = np.zeros(32, dtype=np.uint32)
    nd = np.zeros(1, dtype=np.uint64)
    wi = np.zeros(1, dtype=np.float64)
    wd = np.zeros(1, dtype=np.float64)
    _L().o_float_factor(len(b), _p(b), lam, _p(cnt), _p(nd), _p(wi), _p(wd))
    return cnt, int(nd[0]), float(wi[0]), float(wd[0])
