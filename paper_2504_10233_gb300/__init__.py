"""Python binding of libbingo (radix-factorised biased random walks on dynamic graphs, GB300).

Argument marshalling only: every step of the sampler, the update pipeline and
the walker runs in the library's CUDA kernels.  The functions carry the C ABI's
names (bingo_create, bingo_apply_updates, bingo_walk, ...); `Graph` wraps them.
Arrays may be torch tensors (host or CUDA) or numpy arrays (host); PyTorch is
used only for device memory and streams.  There is no CPU fallback: importing
works without a GPU, but every call needs the built library and a CUDA device.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbingo.so")

OK, E_INVALID, E_OOM, E_CUDA, E_TIMEOUT, E_STATE = range(6)
STATUS_NAMES = {0: "OK", 1: "INVALID", 2: "OOM", 3: "CUDA", 4: "TIMEOUT", 5: "STATE"}
KIND_EMPTY, KIND_DENSE, KIND_ONE, KIND_SPARSE, KIND_REGULAR = range(5)
DEEPWALK, PPR, NODE2VEC = 0, 1, 2
OP_INSERT, OP_DELETE, OP_SET_BIAS = 0, 1, 2
WALK_PERSISTENT, WALK_STEPWISE, WALK_NO_PAD = 0, 1, 0x100
SERVER_NO_MERGE = 1
BIAS_U32, BIAS_F32 = 0, 1
ORDER_AUTO, ORDER_CALLER, ORDER_DEGREE = 0, 1, 2
PAD = 0xFFFFFFFF

c = ctypes
VP = c.c_void_p


class BingoError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"bingo {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class bingo_config(c.Structure):
    _fields_ = [("alpha_pct", c.c_uint32), ("beta_pct", c.c_uint32), ("max_bits", c.c_uint32),
                ("lanes_per_walker", c.c_uint32), ("warps_per_block", c.c_uint32), ("blocks_per_sm", c.c_uint32),
                ("update_chunk", c.c_uint32), ("reg_variant", c.c_uint32), ("pool_words", c.c_uint64),
                ("bias_format", c.c_uint32), ("all_regular", c.c_uint32), ("lambda_", c.c_double),
                ("radix_base", c.c_uint32), ("vertex_order", c.c_uint32), ("vertex_base", c.c_uint32),
                ("dst_space", c.c_uint32), ("hot_l2_hint", c.c_uint32)]


class bingo_update_stats(c.Structure):
    _fields_ = [("inserted", c.c_uint64), ("deleted", c.c_uint64), ("not_found", c.c_uint64),
                ("conversions", (c.c_uint64 * 5) * 5), ("vertices_touched", c.c_uint64),
                ("groups_rebuilt", c.c_uint64)]

    def as_dict(self):
        return {"inserted": self.inserted, "deleted": self.deleted, "not_found": self.not_found,
                "conversions": [[self.conversions[a][b] for b in range(5)] for a in range(5)],
                "vertices_touched": self.vertices_touched, "groups_rebuilt": self.groups_rebuilt}


class bingo_policy(c.Structure):
    _fields_ = [("kind", c.c_uint32), ("max_len", c.c_uint32), ("ppr_stop_u32", c.c_uint32),
                ("reserved", c.c_uint32), ("n2v_accept", c.c_uint64 * 3)]


class bingo_state_sizes(c.Structure):
    _fields_ = [("n", c.c_uint64), ("m", c.c_uint64), ("list_entries", c.c_uint64), ("sparse_entries", c.c_uint64),
                ("pool_words_used", c.c_uint64), ("pool_words_total", c.c_uint64), ("next_edge_id", c.c_uint64)]


class bingo_server_config(c.Structure):
    _fields_ = [("max_inflight_walkers", c.c_uint64), ("hbm_reserve_bytes", c.c_uint64),
                ("max_update_batch", c.c_uint32), ("concurrent_launches", c.c_uint32), ("max_len_cap", c.c_uint32),
                ("flags", c.c_uint32), ("update_delay_us", c.c_uint32), ("reserved", c.c_uint32)]


class bingo_server_request_info(c.Structure):
    _fields_ = [("state", c.c_uint32), ("status", c.c_uint32), ("walkers", c.c_uint64), ("epoch", c.c_uint64),
                ("submit_ms", c.c_double), ("admit_ms", c.c_double), ("done_ms", c.c_double)]


class bingo_server_stats(c.Structure):
    _fields_ = [("requests_done", c.c_uint64), ("walkers_done", c.c_uint64), ("steps_done", c.c_uint64),
                ("updates_applied", c.c_uint64), ("epochs", c.c_uint64), ("p50_ms", c.c_double),
                ("p99_ms", c.c_double), ("mean_ms", c.c_double)]


# name -> (restype, argtypes); this table is also the list of exported symbols the tests check
SIGNATURES = {
    "bingo_version": (c.c_char_p, []),
    "bingo_last_error": (c.c_char_p, []),
    "bingo_default_config": (None, [c.POINTER(bingo_config)]),
    "bingo_create": (c.c_int, [c.c_uint32, c.c_uint64, VP, VP, VP, c.POINTER(bingo_config), VP, c.POINTER(VP)]),
    "bingo_destroy": (c.c_int, [VP]),
    "bingo_apply_updates": (c.c_int, [VP, VP, c.c_uint64, VP, c.POINTER(bingo_update_stats)]),
    "bingo_stream_updates": (c.c_int, [VP, VP, c.c_uint64, VP, c.POINTER(bingo_update_stats)]),
    "bingo_walk": (c.c_int, [VP, c.c_uint64, VP, VP, VP, c.POINTER(bingo_policy), c.c_uint32, c.c_uint64,
                             c.c_uint32, VP, VP, c.c_uint32, VP]),
    "bingo_walk_packed": (c.c_int, [VP, c.c_uint64, VP, VP, VP, c.POINTER(bingo_policy), c.c_uint32, c.c_uint64,
                                    c.c_uint32, VP, VP, c.c_uint64, c.POINTER(c.c_uint64), VP]),
    "bingo_walk_noalloc": (c.c_int, [VP, c.c_uint64, VP, VP, VP, c.POINTER(bingo_policy), c.c_uint32, c.c_uint64,
                                     c.c_uint32, VP, VP, c.c_uint32, VP]),
    "bingo_check": (c.c_int, [VP, VP]),
    "bingo_state_sizes_get": (c.c_int, [VP, c.POINTER(bingo_state_sizes)]),
    "bingo_export_state": (c.c_int, [VP] + [VP] * 13),
    "bingo_export_decimal": (c.c_int, [VP, VP]),
    "bingo_memory_report": (c.c_int, [VP, c.POINTER(c.c_uint64)]),
    "bingo_autotune": (c.c_int, [VP, c.c_uint64, VP, c.c_uint32, VP, c.POINTER(bingo_config)]),
    "bingo_autotune_updates": (c.c_int, [VP, VP, c.c_uint64, VP, c.POINTER(bingo_update_stats), c.POINTER(bingo_config)]),
    "bingo_autotune_adaption": (c.c_int, [c.c_uint32, c.c_uint64, VP, VP, VP, c.POINTER(bingo_config), c.c_uint64,
                                          c.c_uint64, VP, c.c_uint32, VP, c.POINTER(VP), c.POINTER(bingo_config)]),
    "bingo_get_config": (c.c_int, [VP, c.POINTER(bingo_config)]),
    "bingo_set_walk_config": (c.c_int, [VP, c.c_uint32, c.c_uint32, c.c_uint32, c.c_uint32]),
    "bingo_kernel_launches": (c.c_uint64, [VP]),
    "bingo_server_create": (c.c_int, [VP, c.POINTER(bingo_server_config), c.POINTER(VP)]),
    "bingo_server_destroy": (c.c_int, [VP]),
    "bingo_server_submit_updates": (c.c_int, [VP, VP, c.c_uint64, c.POINTER(c.c_uint64)]),
    "bingo_server_submit_walk": (c.c_int, [VP, VP, c.c_uint64, c.POINTER(bingo_policy), c.c_uint64,
                                           c.POINTER(c.c_uint64)]),
    "bingo_server_wait": (c.c_int, [VP, c.c_uint64, c.c_uint32, VP, VP, c.POINTER(c.c_uint64)]),
    "bingo_server_drain": (c.c_int, [VP, c.c_uint32]),
    "bingo_server_stats_get": (c.c_int, [VP, c.POINTER(bingo_server_stats)]),
    "bingo_server_pause": (c.c_int, [VP, c.c_uint32]),
    "bingo_server_request_get": (c.c_int, [VP, c.c_uint64, c.POINTER(bingo_server_request_info)]),
    "bingo_export_vertices_sizes": (c.c_int, [VP, VP, c.c_uint64, c.POINTER(c.c_uint64)]),
    "bingo_export_vertices": (c.c_int, [VP, VP, c.c_uint64] + [VP] * 13),
    "bingo_part_create": (c.c_int, [c.c_uint32, c.c_uint64, VP, VP, VP, c.POINTER(bingo_config), c.c_uint32, VP, VP,
                                    c.POINTER(VP)]),
    "bingo_part_destroy": (c.c_int, [VP]),
    "bingo_part_info": (c.c_int, [VP, c.c_uint32, c.POINTER(VP), c.POINTER(c.c_uint32), c.POINTER(c.c_uint32)]),
    "bingo_part_apply_updates": (c.c_int, [VP, VP, c.c_uint64, VP, c.POINTER(bingo_update_stats)]),
    "bingo_part_walk": (c.c_int, [VP, c.c_uint64, VP, VP, VP, c.POINTER(bingo_policy), c.c_uint32, c.c_uint64,
                                  c.c_uint32, VP, VP, c.c_uint32, VP]),
    "bingo_part_check": (c.c_int, [VP, VP]),
    "bingo_part_supersteps": (c.c_uint64, [VP]),
    "bingo_policy_make": (c.c_int, [c.c_uint32, c.c_uint32, c.c_double, c.c_double, c.c_double,
                                    c.POINTER(bingo_policy)]),
    "bingo_philox4x32_10": (c.c_int, [c.c_uint64, VP, VP, VP]),
    "bingo_walker_draws": (c.c_int, [c.c_uint64, c.c_uint64, c.c_uint32, c.c_uint64, c.c_uint32, VP]),
}

_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return LIB_PATH


def load():
    """Load libbingo.so; raise if it is missing (run __graft_entry__.build() or _build.build())."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(f"libbingo.so not built at {LIB_PATH}; the CUDA path is required")
            lib = c.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def _err(st: int):
    if st != OK:
        raise BingoError(st, load().bingo_last_error().decode(errors="replace"))


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        assert x.flags["C_CONTIGUOUS"], "arrays must be contiguous"
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        assert x.is_contiguous(), "tensors must be contiguous"
        return x.data_ptr()
    if isinstance(x, int):
        return x
    raise TypeError(f"unsupported buffer type {type(x)}")


def _stream(s):
    if s is None:
        return None
    if hasattr(s, "cuda_stream"):
        return s.cuda_stream
    return int(s)


def policy(kind: int, max_len: int, ppr_stop: float | int = 0, n2v_pq=None) -> bingo_policy:
    """Walk policy through bingo_policy_make.  ppr_stop: probability (float) or u32 threshold (int).
    n2v_pq = (p, q) for node2vec."""
    p = bingo_policy()
    pp, qq = n2v_pq if n2v_pq is not None else (1.0, 1.0)
    prob = float(ppr_stop) if isinstance(ppr_stop, float) else 0.0
    _err(load().bingo_policy_make(kind, max_len, prob, float(pp), float(qq), c.byref(p)))
    if not isinstance(ppr_stop, float):
        p.ppr_stop_u32 = int(ppr_stop)
    return p


def bingo_philox4x32_10(ctr, key) -> np.ndarray:
    """Philox4x32-10 evaluated on the device by the walker's own code: ctr u32[count, 4], key u32[count, 2]."""
    ctr = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32).reshape(-1, 4))
    key = np.ascontiguousarray(np.asarray(key, dtype=np.uint32).reshape(-1, 2))
    assert len(ctr) == len(key)
    out = np.zeros_like(ctr)
    _err(load().bingo_philox4x32_10(len(ctr), _ptr(ctr), _ptr(key), _ptr(out)))
    return out


def bingo_walker_draws(seed: int, walker: int, step: int, count: int, range_: int = 0) -> np.ndarray:
    """The draws walker `walker` makes at step `step` under key `seed` (raw u32 words, or bounded in
    [0, range_) when range_ >= 1), evaluated on the device."""
    out = np.zeros(count, dtype=np.uint64)
    _err(load().bingo_walker_draws(int(seed), int(walker), int(step), int(range_), int(count), _ptr(out)))
    return out


def default_config(max_bits: int = 32, **kw) -> bingo_config:
    cfg = bingo_config()
    load().bingo_default_config(c.byref(cfg))
    cfg.max_bits = max_bits
    for k, v in kw.items():
        setattr(cfg, k, v)
    return cfg


# ------------------------------------------------------------------------------------- same-name wrappers


def bingo_create(n, row_ptr, col, bias, cfg=None, stream=None):
    h = VP()
    m = int(len(col))
    st = load().bingo_create(n, m, _ptr(row_ptr), _ptr(col), _ptr(bias), c.byref(cfg) if cfg is not None else None,
                             _stream(stream), c.byref(h))
    _err(st)
    return h


def bingo_destroy(h):
    _err(load().bingo_destroy(h))


def bingo_apply_updates(h, records, count=None, stream=None):
    stats = bingo_update_stats()
    count = int(records.shape[0]) if count is None else count
    _err(load().bingo_apply_updates(h, _ptr(records), count, _stream(stream), c.byref(stats)))
    return stats.as_dict()


def bingo_stream_updates(h, records, count=None, stream=None):
    stats = bingo_update_stats()
    count = int(records.shape[0]) if count is None else count
    _err(load().bingo_stream_updates(h, _ptr(records), count, _stream(stream), c.byref(stats)))
    return stats.as_dict()


def bingo_walk(h, nwalkers, starts, policies, seed, stride, paths, path_len, lengths=None, policy_ids=None,
               mode=WALK_PERSISTENT, stream=None):
    arr = (bingo_policy * len(policies))(*policies)
    _err(load().bingo_walk(h, nwalkers, _ptr(starts), _ptr(lengths), _ptr(policy_ids), arr, len(policies), seed,
                           stride, _ptr(paths), _ptr(path_len), mode, _stream(stream)))


def bingo_walk_packed(h, nwalkers, starts, policies, seed, max_steps, path_len, vertices, lengths=None,
                      policy_ids=None, stream=None) -> int:
    """Packed walk (no padding): returns the number of vertices written to `vertices`."""
    arr = (bingo_policy * len(policies))(*policies)
    tot = c.c_uint64()
    cap = int(vertices.numel() if hasattr(vertices, "numel") else vertices.size)
    _err(load().bingo_walk_packed(h, nwalkers, _ptr(starts), _ptr(lengths), _ptr(policy_ids), arr, len(policies),
                                  seed, max_steps, _ptr(path_len), _ptr(vertices), cap, c.byref(tot), _stream(stream)))
    return int(tot.value)


def bingo_walk_noalloc(h, nwalkers, starts, policies, seed, stride, paths, path_len, lengths=None, policy_ids=None,
                       mode=WALK_PERSISTENT, stream=None):
    """bingo_walk without any device allocation (device buffers only; see include/bingo.h)."""
    arr = (bingo_policy * len(policies))(*policies)
    _err(load().bingo_walk_noalloc(h, nwalkers, _ptr(starts), _ptr(lengths), _ptr(policy_ids), arr, len(policies),
                                   seed, stride, _ptr(paths), _ptr(path_len), mode, _stream(stream)))


def bingo_check(h, stream=None):
    _err(load().bingo_check(h, _stream(stream)))


def bingo_memory_report(h):
    out = (c.c_uint64 * 6)()
    _err(load().bingo_memory_report(h, out))
    keys = ["adjacency", "vertex_records", "regular_groups", "sparse_groups", "edge_index", "pool_capacity"]
    return dict(zip(keys, [int(x) for x in out]))


def bingo_autotune_updates(h, records, stream=None):
    """Tune update_chunk on these records, which are applied (as consecutive slices)."""
    cfg = bingo_config()
    st = bingo_update_stats()
    n = int(records.shape[0]) if hasattr(records, "shape") else len(records)
    _err(load().bingo_autotune_updates(h, _ptr(records), n, _stream(stream), c.byref(st), c.byref(cfg)))
    return st.as_dict(), cfg


def bingo_autotune(h, nwalkers, starts, length, stream=None):
    cfg = bingo_config()
    _err(load().bingo_autotune(h, nwalkers, _ptr(starts), length, _stream(stream), c.byref(cfg)))
    return cfg


def bingo_autotune_adaption(n, row_ptr, col, bias, cfg, state_budget_bytes, starts, length, stream=None):
    """Build the graph under each candidate (alpha, beta) and keep the fastest within the budget;
    returns (handle, chosen config)."""
    h = VP()
    out = bingo_config()
    _err(load().bingo_autotune_adaption(n, int(len(col)), _ptr(row_ptr), _ptr(col), _ptr(bias),
                                        c.byref(cfg) if cfg is not None else None, int(state_budget_bytes),
                                        int(len(starts)), _ptr(starts), length, _stream(stream), c.byref(h),
                                        c.byref(out)))
    return h, out


def state_sizes(h) -> dict:
    """bingo_state_sizes_get as a dict (n, m, list_entries, sparse_entries, pool words, next edge id)."""
    sz = bingo_state_sizes()
    _err(load().bingo_state_sizes_get(h, c.byref(sz)))
    return {f: int(getattr(sz, f)) for f, _ in bingo_state_sizes._fields_}


def _size_class(x: int) -> int:
    return max(0, int(x) - 1).bit_length()  # ceil(log2 x): graphs within a factor of two share a class


def walk_tune_key(graph, length: int, device: str) -> str:
    """Cache key of a tuned walker launch: the device, the graph's size class and weight format, the walk length."""
    cfg = graph.config()
    m = graph.state_sizes()["m"]
    return (f"{device}|n2^{_size_class(graph.n)}|m2^{_size_class(m)}|bits{cfg.max_bits}|fmt{cfg.bias_format}"
            f"|base{cfg.radix_base or 2}|L{int(length)}")


def cached_walk_tune(graph, starts, length: int, cache_path: str, device: str, stream=None) -> dict:
    """The walker launch shape (lanes per walker, warps per block, blocks per SM, register variant) from a
    JSON cache keyed by walk_tune_key; on a miss bingo_autotune measures it on `starts` and the result is
    stored (the file is replaced atomically).  Returns the shape and whether it came from the cache."""
    import json

    key = walk_tune_key(graph, length, device)
    data = {"version": 1, "entries": {}}
    if os.path.exists(cache_path):
        with open(cache_path) as fh:
            data = json.load(fh)
    fields = ("lanes_per_walker", "warps_per_block", "blocks_per_sm", "reg_variant")
    hit = data.get("entries", {}).get(key)
    if hit is not None:
        graph.set_walk_config(hit["lanes_per_walker"], hit["warps_per_block"], hit["blocks_per_sm"],
                              hit["reg_variant"])
        return dict(hit, cached=True)
    cfg = graph.autotune(starts, length, stream=stream)
    entry = {f: int(getattr(cfg, f)) for f in fields}
    data.setdefault("entries", {})[key] = entry
    tmp = f"{cache_path}.tmp{os.getpid()}"
    with open(tmp, "w") as fh:
        json.dump(data, fh, indent=1, sort_keys=True)
    os.replace(tmp, cache_path)
    return dict(entry, cached=False)


def bingo_get_config(h):
    cfg = bingo_config()
    _err(load().bingo_get_config(h, c.byref(cfg)))
    return cfg


def bingo_set_walk_config(h, lanes, warps_per_block, blocks_per_sm=0, reg_variant=0):
    _err(load().bingo_set_walk_config(h, lanes, warps_per_block, blocks_per_sm, reg_variant))


def bingo_kernel_launches(h) -> int:
    return int(load().bingo_kernel_launches(h))


def bingo_export_state(h):
    """Whole sampling state as numpy arrays (see bingo_export_state in include/bingo.h)."""
    L = load()
    sz = bingo_state_sizes()
    _err(L.bingo_state_sizes_get(h, c.byref(sz)))
    n, m, le, se = sz.n, sz.m, sz.list_entries, sz.sparse_entries
    out = {
        "deg": np.zeros(n, np.uint32), "dst": np.zeros(max(m, 1), np.uint32), "bias": np.zeros(max(m, 1), np.uint32),
        "eid": np.zeros(max(m, 1), np.uint64), "cnt": np.zeros(32 * n, np.uint32), "kind": np.zeros(32 * n, np.uint8),
        "one_slot": np.zeros(32 * n, np.uint32), "glen": np.zeros(32 * n, np.uint32),
        "members": np.zeros(max(le, 1), np.uint32), "member_inv": np.zeros(max(le, 1), np.uint32),
        "sp_len": np.zeros(n, np.uint32), "sp_list": np.zeros(max(se, 1), np.uint32),
        "sp_inv": np.zeros(max(se, 1), np.uint32),
    }
    order = ["deg", "dst", "bias", "eid", "cnt", "kind", "one_slot", "glen", "members", "member_inv", "sp_len",
             "sp_list", "sp_inv"]
    _err(L.bingo_export_state(h, *[_ptr(out[k]) for k in order]))
    for k in ("dst", "bias", "eid"):
        out[k] = out[k][:m]
    out["members"], out["member_inv"] = out["members"][:le], out["member_inv"][:le]
    out["sp_list"], out["sp_inv"] = out["sp_list"][:se], out["sp_inv"][:se]
    out["cnt"] = out["cnt"].reshape(n, 32)
    out["kind"] = out["kind"].reshape(n, 32)
    out["one_slot"] = out["one_slot"].reshape(n, 32)
    out["glen"] = out["glen"].reshape(n, 32)
    out["sizes"] = {f: getattr(sz, f) for f, _ in bingo_state_sizes._fields_}
    return out


def bingo_export_vertices(h, ids):
    """The state of the listed caller vertices (row i = ids[i]) in the layout of bingo_export_state."""
    L = load()
    ids = np.ascontiguousarray(np.asarray(ids, dtype=np.uint32))
    k = len(ids)
    sz = (c.c_uint64 * 3)()
    _err(L.bingo_export_vertices_sizes(h, _ptr(ids), k, sz))
    m, le, se = int(sz[0]), int(sz[1]), int(sz[2])
    out = {
        "deg": np.zeros(k, np.uint32), "dst": np.zeros(max(m, 1), np.uint32), "bias": np.zeros(max(m, 1), np.uint32),
        "eid": np.zeros(max(m, 1), np.uint64), "cnt": np.zeros(32 * k, np.uint32), "kind": np.zeros(32 * k, np.uint8),
        "one_slot": np.zeros(32 * k, np.uint32), "glen": np.zeros(32 * k, np.uint32),
        "members": np.zeros(max(le, 1), np.uint32), "member_inv": np.zeros(max(le, 1), np.uint32),
        "sp_len": np.zeros(k, np.uint32), "sp_list": np.zeros(max(se, 1), np.uint32),
        "sp_inv": np.zeros(max(se, 1), np.uint32),
    }
    order = ["deg", "dst", "bias", "eid", "cnt", "kind", "one_slot", "glen", "members", "member_inv", "sp_len",
             "sp_list", "sp_inv"]
    _err(L.bingo_export_vertices(h, _ptr(ids), k, *[_ptr(out[x]) for x in order]))
    for x in ("dst", "bias", "eid"):
        out[x] = out[x][:m]
    out["members"], out["member_inv"] = out["members"][:le], out["member_inv"][:le]
    out["sp_list"], out["sp_inv"] = out["sp_list"][:se], out["sp_inv"][:se]
    for x in ("cnt", "kind", "one_slot", "glen"):
        out[x] = out[x].reshape(k, 32)
    out["ids"] = ids
    return out


def bingo_export_decimal(h):
    """Decimal parts (units of 2^-8) of every live edge of a real-bias graph, in export order."""
    L = load()
    sz = bingo_state_sizes()
    _err(L.bingo_state_sizes_get(h, c.byref(sz)))
    q = np.zeros(max(sz.m, 1), np.uint8)
    _err(L.bingo_export_decimal(h, _ptr(q)))
    return q[: sz.m]


def real_bias_bits(b) -> np.ndarray:
    """binary32 encodings of real biases, the bias words of a BIAS_F32 graph or update."""
    return np.ascontiguousarray(np.asarray(b, dtype=np.float32)).view(np.uint32)


# ------------------------------------------------------------------------------------- object wrapper


class Graph:
    """Owns a bingo_graph.  Thin: every method is one C-ABI call."""

    def __init__(self, n, row_ptr, col, bias, max_bits=32, stream=None, **cfg):
        self.n = int(n)
        self.cfg = default_config(max_bits=max_bits, **cfg)
        self.h = bingo_create(self.n, row_ptr, col, bias, self.cfg, stream)

    @classmethod
    def tuned(cls, n, row_ptr, col, bias, starts, length, state_budget_bytes=0, max_bits=32, stream=None, **cfg):
        """A graph whose group-adaption thresholds were chosen by bingo_autotune_adaption."""
        self = cls.__new__(cls)
        self.n = int(n)
        base = default_config(max_bits=max_bits, **cfg)
        self.h, self.cfg = bingo_autotune_adaption(self.n, row_ptr, col, bias, base, state_budget_bytes, starts,
                                                   length, stream)
        return self

    def close(self):
        if getattr(self, "h", None):
            bingo_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def apply_updates(self, records, stream=None):
        return bingo_apply_updates(self.h, records, stream=stream)

    def stream_updates(self, records, stream=None):
        return bingo_stream_updates(self.h, records, stream=stream)

    def walk(self, starts, policies, seed, stride, paths, path_len, lengths=None, policy_ids=None,
             mode=WALK_PERSISTENT, stream=None):
        bingo_walk(self.h, len(starts), starts, policies, seed, stride, paths, path_len, lengths, policy_ids, mode,
                   stream)

    def walk_packed(self, starts, policies, seed, max_steps, path_len, vertices, lengths=None, policy_ids=None,
                    stream=None) -> int:
        return bingo_walk_packed(self.h, len(starts), starts, policies, seed, max_steps, path_len, vertices, lengths,
                                 policy_ids, stream)

    def check(self, stream=None):
        bingo_check(self.h, stream)

    def export_state(self):
        return bingo_export_state(self.h)

    def export_vertices(self, ids):
        return bingo_export_vertices(self.h, ids)

    def export_decimal(self):
        return bingo_export_decimal(self.h)

    def memory_report(self):
        return bingo_memory_report(self.h)

    def autotune(self, starts, length, stream=None):
        return bingo_autotune(self.h, len(starts), starts, length, stream)

    def autotune_updates(self, records, stream=None):
        return bingo_autotune_updates(self.h, records, stream)

    def set_walk_config(self, lanes, warps_per_block, blocks_per_sm=0, reg_variant=0):
        bingo_set_walk_config(self.h, lanes, warps_per_block, blocks_per_sm, reg_variant)

    def config(self):
        return bingo_get_config(self.h)

    def state_sizes(self) -> dict:
        return state_sizes(self.h)

    def cached_walk_tune(self, starts, length, cache_path, device, stream=None) -> dict:
        return cached_walk_tune(self, starts, length, cache_path, device, stream)

    def kernel_launches(self) -> int:
        return bingo_kernel_launches(self.h)


class PartitionedGraph:
    """Owns a bingo_partset: the graph split into vertex ranges, walked with walker migration."""

    def __init__(self, n, row_ptr, col, bias, nparts, bounds=None, max_bits=32, stream=None, **cfg):
        self.n = int(n)
        self.cfg = default_config(max_bits=max_bits, **cfg)
        h = VP()
        b = None if bounds is None else np.ascontiguousarray(np.asarray(bounds, dtype=np.uint32))
        _err(load().bingo_part_create(self.n, int(len(col)), _ptr(row_ptr), _ptr(col), _ptr(bias), c.byref(self.cfg),
                                      int(nparts), _ptr(b), _stream(stream), c.byref(h)))
        self.h = h
        self.nparts = int(nparts)

    def close(self):
        if getattr(self, "h", None):
            load().bingo_part_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def part(self, p):
        """(partition graph handle, lo, hi) of partition p."""
        g, lo, hi = VP(), c.c_uint32(), c.c_uint32()
        _err(load().bingo_part_info(self.h, p, c.byref(g), c.byref(lo), c.byref(hi)))
        return g, int(lo.value), int(hi.value)

    def export_vertices(self, p, local_ids):
        return bingo_export_vertices(self.part(p)[0], local_ids)

    def apply_updates(self, records, stream=None):
        stats = bingo_update_stats()
        _err(load().bingo_part_apply_updates(self.h, _ptr(records), int(records.shape[0]), _stream(stream),
                                             c.byref(stats)))
        return stats.as_dict()

    def walk(self, starts, policies, seed, stride, paths, path_len, lengths=None, policy_ids=None,
             mode=WALK_PERSISTENT, stream=None):
        arr = (bingo_policy * len(policies))(*policies)
        _err(load().bingo_part_walk(self.h, len(starts), _ptr(starts), _ptr(lengths), _ptr(policy_ids), arr,
                                    len(policies), seed, stride, _ptr(paths), _ptr(path_len), mode, _stream(stream)))

    def check(self, stream=None):
        _err(load().bingo_part_check(self.h, _stream(stream)))

    def supersteps(self) -> int:
        return int(load().bingo_part_supersteps(self.h))
