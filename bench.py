"""Benchmark: sampled walk steps/s and updated edges/s on one GB300 (and N replicas).

Workload (default): RMAT scale 20 (2^20 vertices, 2^24 edges, a=.57 b=.19 c=.19),
biases floor(Pareto(1.5)) clipped to 2^20; one step = one batch of 10^5 edge
updates (50% insert / 50% delete, the paper's hold-out protocol) applied in
place, then 2^20 biased DeepWalk walkers of length 80 from uniform starts.
`value` = sampled steps / (update + walk time) over the timed steps, device
timed with CUDA events; updates/s and walk-only steps/s are reported beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload c2]

Under torchrun each rank runs an independent replica (walker seeds differ by
rank); value = all ranks' steps / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

PEAKS_FALLBACK = {"hbm_gbs": 6800.0}
L2_FLUSH_BYTES = 512 << 20


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return PEAKS_FALLBACK, "fallback"


# ------------------------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every PERIOD_MS from before the warm-up (starting the
    sampler costs seconds, which must not fall in the timed region); stop() keeps the samples read
    inside the timed window [mark_start(), mark_end()]."""

    # While nvidia-smi runs, this process's host time over the timed steps grows by about 2.5 s
    # (7 RMAT-20 steps of 2.3 ms: 2.46 s of wall at 200 ms polling, 2.52 s at 1,000 ms, 0.02 s
    # without the sampler); the events, and so the value, do not see it
    PERIOD_MS = 200
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []
        self.t0 = self.t1 = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", str(self.PERIOD_MS)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def wait_first(self, timeout=15.0):
        """Block until nvidia-smi has printed its first sample: its start-up (NVML initialisation) holds
        driver locks that stall CUDA calls, and must not overlap the timed region."""
        t_end = time.perf_counter() + timeout
        while self.proc is not None and not self.lines and time.perf_counter() < t_end:
            time.sleep(0.05)

    def mark_start(self):
        self.t0 = time.perf_counter()

    def mark_end(self):
        self.t1 = time.perf_counter()

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        if self.t1 is not None:  # one more sample period so the window's last sample is read
            while time.perf_counter() < self.t1 + self.PERIOD_MS / 1e3 + 0.05:
                time.sleep(0.05)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        lo = self.t0 if self.t0 is not None else -1e300
        hi = (self.t1 + self.PERIOD_MS / 1e3 + 0.05) if self.t1 is not None else 1e300
        inside = [ln for ts, ln in self.lines if lo <= ts <= hi]
        if not inside and self.lines:  # a window shorter than the sampling period: the nearest sample
            mid = 0.5 * (lo + hi) if self.t0 is not None and self.t1 is not None else self.lines[-1][0]
            inside = [min(self.lines, key=lambda x: abs(x[0] - mid))[1]]
        for ln in inside:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for nm, val in zip(names, f[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------------------------- roofline model

WALK_SOURCES = ["paper_2504_10233_gb300/csrc/walk.cu", "paper_2504_10233_gb300/csrc/bingo_internal.cuh"]


def walk_source_digest() -> str:
    import hashlib

    h = hashlib.sha256()
    for f in WALK_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic(workload: str):
    """DRAM bytes (read + write) per walker launch from the committed ncu capture of this workload,
    or None when the walker sources changed since the capture (the digest no longer matches)."""
    path = os.path.join(ROOT, "profiles", "walk_traffic.json")
    try:
        with open(path) as fh:
            rec = json.load(fh)
    except (OSError, ValueError):
        return None
    ent = rec.get(workload)
    if not ent or ent.get("sources_sha256_16") != walk_source_digest():
        return None
    return float(ent["dram_bytes_per_launch"])

def expected_bytes_per_vertex(ex, alpha=40, beta=10):
    """Algorithmic bytes of one sampled step from each vertex, averaged over the group choice:
    header sector 32 + count line 32*ceil(4*K_v/32) + the group's pick (regular: member sector 32,
    sparse: + sparse-list sector 32, one-element: stored index, dense: 32 per rejection trial with
    E[trials] = d/|G_k|; the target edge sector 32 for non-dense picks) + 4 bytes of path output."""
    deg = ex["deg"].astype(np.float64)
    cnt = ex["cnt"].astype(np.float64)
    kind = ex["kind"]
    k = np.arange(32, dtype=np.float64)
    Wk = cnt * np.exp2(k)[None, :]
    tot = Wk.sum(axis=1)
    mask = cnt > 0
    kv = np.where(mask.any(axis=1), 32 - np.argmax(mask[:, ::-1], axis=1), 0)
    line = 32.0 * np.ceil(4.0 * kv / 32.0)
    with np.errstate(divide="ignore", invalid="ignore"):
        p = np.where(tot[:, None] > 0, Wk / tot[:, None], 0.0)
        trials = np.where(cnt > 0, deg[:, None] / np.maximum(cnt, 1), 0.0)
    cost = np.zeros_like(cnt)
    cost = np.where(kind == 1, 32.0 * trials, cost)      # dense: each trial reads one {dst, bias} sector
    cost = np.where(kind == 2, 32.0, cost)               # one-element: target edge
    cost = np.where(kind == 4, 64.0, cost)               # regular: member + target
    cost = np.where(kind == 3, 96.0, cost)               # sparse: member + sparse list + target
    per = 32.0 + line + (p * cost).sum(axis=1) + 4.0
    return np.where(deg > 0, per, 0.0)


def expected_bytes_parts(ex):
    """The per-vertex model split into what a step reads once (header sector, count line) and what
    every draw of a candidate reads again (the group's pick), for walks that retry candidates."""
    deg = ex["deg"].astype(np.float64)
    cnt = ex["cnt"].astype(np.float64)
    mask = cnt > 0
    kv = np.where(mask.any(axis=1), 32 - np.argmax(mask[:, ::-1], axis=1), 0)
    fixed = np.where(deg > 0, 32.0 + 32.0 * np.ceil(4.0 * kv / 32.0), 0.0)
    pick = np.where(deg > 0, expected_bytes_per_vertex(ex) - fixed - 4.0, 0.0)
    return fixed, pick


def node2vec_step_bytes(fixed, pick, p_accept, p_probe, probe_bytes=64.0):
    """Model bytes of one node2vec step by rejection (Eq. node2vec): the step's fixed part once, then
    E[candidates] = 1 / P(accept) picks, each followed with probability p_probe by an edge-index probe
    (the key's sector and its count's), and the 4-byte path entry."""
    return fixed + (pick + p_probe * probe_bytes) / p_accept + 4.0


def walk_bytes(per_vertex, paths, plen):
    """Sum of per-step bytes over the recorded walks (steps leave from paths[:, t], t < plen-1)."""
    L = paths.shape[1]
    valid = np.arange(L - 1)[None, :] < (plen.astype(np.int64)[:, None] - 1)
    src = paths[:, :-1][valid].astype(np.int64)
    return float(per_vertex[src].sum())


def sample_steps(plen, k, seed):
    """k steps drawn uniformly (with replacement) from all sampled steps of a launch: (walker, t) with
    t < plen - 1; the step leaves from path entry t."""
    steps = np.maximum(plen.astype(np.int64) - 1, 0)
    cum = np.cumsum(steps)
    tot = int(cum[-1]) if len(cum) else 0
    if tot == 0:
        return np.zeros(0, np.int64), np.zeros(0, np.int64), 0
    u = np.random.default_rng(seed).integers(0, tot, size=k)
    w = np.searchsorted(cum, u, side="right")
    t = u - (cum[w] - steps[w])
    return w, t, tot


def update_bytes(ex0, ex1, rec, ids=None):
    """Algorithmic bytes of one update batch, from the exported state before (ex0) and after (ex1) it:
    per record its 16 bytes and a sort by source (two passes of 16 bytes read + 16 written); per
    insertion the adjacency slot (32) and, for every set bit k whose group (v, k) is a member list
    (regular or sparse) after the batch, the member entry and its inverted-index entry (32 + 32);
    per deletion that finds its edge the locating probe (32), the adjacency slot (32), one compaction
    move (32), and for every set bit of the removed edge whose group was a list before the batch the
    entry, its inverted entry, the tail read and the patch (4 x 32); per touched vertex its count line
    read and written (2 x 32 ceil(4 K_v / 32), K_v = highest nonempty group + 1 after the batch).
    ids: when the exports hold only some vertices (bingo_export_vertices), the sorted vertex of each
    row; they must include every source of the batch."""
    rec = np.asarray(rec, dtype=np.uint32).reshape(-1, 4)
    src = rec[:, 0].astype(np.int64)
    if ids is not None:
        ids = np.asarray(ids, dtype=np.int64)
        row = np.searchsorted(ids, src)
        assert (ids[np.minimum(row, len(ids) - 1)] == src).all(), "every source needs an exported row"
        src = row
    op = rec[:, 3]
    ins, dele = op != 1, op != 0
    nbytes = 16.0 * len(rec) + 64.0 * float(ins.sum() + dele.sum())
    sh = np.arange(32, dtype=np.uint64)
    # insertions
    k1 = ex1["kind"]
    listk1 = (k1 == 3) | (k1 == 4)
    bits = ((rec[ins, 2].astype(np.uint64)[:, None] >> sh[None, :]) & np.uint64(1)).astype(bool)
    nbytes += 32.0 * float(ins.sum()) + 64.0 * float((bits & listk1[src[ins]]).sum())
    # deletions: the earliest live copy of (src, dst) before the batch
    deg0 = ex0["deg"].astype(np.int64)
    v0 = np.repeat(np.arange(len(deg0), dtype=np.uint64), deg0)
    key0 = (v0 << np.uint64(32)) | ex0["dst"].astype(np.uint64)
    order = np.lexsort((ex0["eid"], key0))
    key0s, bias0s = key0[order], ex0["bias"][order]
    first = np.ones(len(key0s), dtype=bool)
    first[1:] = key0s[1:] != key0s[:-1]
    key0s, bias0s = key0s[first], bias0s[first]
    dk = (src[dele].astype(np.uint64) << np.uint64(32)) | rec[dele, 1].astype(np.uint64)
    pos = np.minimum(np.searchsorted(key0s, dk), max(len(key0s) - 1, 0))
    found = (key0s[pos] == dk) if len(key0s) else np.zeros(len(dk), dtype=bool)
    listk0 = (ex0["kind"] == 3) | (ex0["kind"] == 4)
    dbits = ((bias0s[pos[found]].astype(np.uint64)[:, None] >> sh[None, :]) & np.uint64(1)).astype(bool)
    nbytes += 96.0 * float(found.sum()) + 128.0 * float((dbits & listk0[src[dele][found]]).sum())
    # touched vertices
    tv = np.unique(src)
    mask1 = ex1["cnt"][tv] > 0
    kv = np.where(mask1.any(axis=1), 32 - np.argmax(mask1[:, ::-1], axis=1), 0)
    nbytes += float((2.0 * 32.0 * np.ceil(4.0 * kv / 32.0)).sum())
    return nbytes


# ------------------------------------------------------------------------------------- distributed helpers

def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x: float, backend_device=None) -> float:
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        return x
    t = torch.tensor([x], dtype=torch.float64, device=backend_device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, backend_device=None) -> float:
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        return x
    t = torch.tensor([x], dtype=torch.float64, device=backend_device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def replica_seed(base: int, rank: int) -> int:
    """Each replica walks with its own Philox key so replicas sample independent walks."""
    return base + 0x9E3779B97F4A7C15 * rank & 0xFFFFFFFFFFFFFFFF


# ------------------------------------------------------------------------------------- workloads of the main line

SWEEP_SIZES = [10 ** e for e in range(3, 8)]
SWEEP_REPS = 3  # per size: one untimed batch (capacity growth and graph capture happen there), two timed

MAIN = {
    # RMAT-26 + 64 hubs, uniform 31-bit biases: per step a 10^6-record batch, then 16M PPR walkers
    "c5": dict(policy="ppr", length=100, ppr_stop=0.15, batch=10 ** 6, sweep=True,
               text="RMAT-26 (2^26 vertices, 2^30 edges) + 64 hubs x 10^6 extra out-edges, uniform biases in "
                    "[1, 2^31); per step: 10^6 updates (50/50, hold-out protocol) then 16M PPR walkers "
                    "(stop 0.15, cap 100)"),
    # ER 1,024 / 16,384, biases U[1, 255]: per step a batch of 1,024 inserts + 1,024 deletes, then 1,024
    # DeepWalk walkers x 80 (a correctness workload: its state fits L2)
    "c1": dict(policy="deepwalk", length=80, ppr_stop=0.0, batch=2048, sweep=False,
               text="ER directed (1,024 vertices, 16,384 edges), biases U[1, 255]; per step: 1,024 inserts + 1,024 "
                    "deletes then 1,024 DeepWalk walkers x 80"),
    # RMAT-20, floor(Pareto 1.5) biases: per step a 10^5-record batch, then 2^20 DeepWalk walkers x 80
    "c2": dict(policy="deepwalk", length=80, ppr_stop=0.0, batch=10 ** 5, sweep=False,
               text="RMAT-20 (2^20 vertices, 2^24 edges, a=.57 b=.19 c=.19), floor(Pareto 1.5) biases <= 2^20; "
                    "per step: 10^5 updates (50/50) then 2^20 DeepWalk walkers x 80"),
}

POLICY_NAME = {"deepwalk": "DeepWalk", "ppr": "PPR (stop 0.15; x = cap)"}

METRIC_MAIN = "sampled walk steps/s (update batch + walk per step); updated edges/s; p50/p99 latency in the serving bench"


def main_workload(name, nsteps, scale=None, hubs=True, nwalkers=None):
    """The workload and its per-step batches (plus, for c5, the records of the batch-size sweep): one
    stream of hold-out-protocol records cut into consecutive batches.  scale: a smaller RMAT scale of
    the same recipe (edge factor 16; hubs keep their degree up to a sixteenth of the edges), for
    profiling captures that must stay small."""
    spec = MAIN[name]
    extra = SWEEP_REPS * sum(SWEEP_SIZES) if spec["sweep"] else 0
    shrink = {} if scale is None else {"scale": scale, "m": 16 << scale}
    if not hubs:
        shrink["hubs"] = False
    if nwalkers:
        shrink["nwalkers"] = nwalkers
    if name in ("c1", "c2"):
        wl = W.make_workload(name, nbatch=nsteps, **shrink)
        return wl, [b.records() for b in wl.batches], None
    wl = W.make_workload(name, nbatch=1, batch=nsteps * spec["batch"] + extra, **shrink)
    rec = wl.batches[0].records()
    b = spec["batch"]
    return wl, [rec[i * b:(i + 1) * b] for i in range(nsteps)], rec[nsteps * b:]


def main_config(args, wl, name=None):
    """The workload part of the main line's config, shared by both arms."""
    name = name or args.workload
    spec = MAIN[name]
    text = spec["text"]
    if getattr(args, "scale", None) is not None and name == args.workload:
        text = f"scaled to RMAT-{args.scale} (2^{args.scale} vertices, edge factor 16), otherwise: " + text
    if getattr(args, "no_hubs", False) and name == args.workload:
        text = "without its hub edges (profiling), otherwise: " + text
    if getattr(args, "walkers", None) and name == args.workload:
        text = f"{args.walkers} walkers per step (profiling), otherwise: " + text
    return {"workload": text, "walkers": wl.nwalkers, "length": spec["length"], "policy": spec["policy"],
            "updates_per_step": spec["batch"]}


def _oracle_policy(O, name):
    spec = MAIN[name]
    if spec["policy"] == "ppr":
        return O.policy(O.PPR, spec["length"], int(round(spec["ppr_stop"] * 2 ** 32)))
    return O.policy(O.DEEPWALK, spec["length"])


# ------------------------------------------------------------------------------------- CPU baseline

def cpu_baseline(G, batch, length, seed, target_s=15.0, name="c2", one_thread_s=None):
    """The oracle as it stands, on a bounded sample: the first update batch applied, then as many
    walkers of the workload's policy as fit in about target_s seconds (calibrated on a small run), on
    all host cores; with one_thread_s, the same at one thread on a sample sized for about that long."""
    import oracle as O

    og = O.Graph(G.n, G.row_ptr, G.col, G.w)
    rec = batch.records() if hasattr(batch, "records") else batch
    t0 = time.perf_counter()
    og.apply(rec, G.max_bits)
    t_apply = time.perf_counter() - t0
    pol = _oracle_policy(O, name)
    cores = O.num_threads()

    def timed(nw, seed_):
        st = W.walk_starts(G.n, nw, seed_)
        t0 = time.perf_counter()
        _, plen = og.walk(st, [pol], seed_)
        return float((plen.astype(np.int64) - 1).sum()), time.perf_counter() - t0

    def sized(budget_s, seed_):
        # every walk call first rebuilds the prefix sums of the whole graph: fit that fixed cost and
        # the cost per walker from two calibration calls, then size the sample to the budget
        _, t1 = timed(4096, seed_)
        _, t2 = timed(32768, seed_ + 2)
        per = max((t2 - t1) / (32768 - 4096), 1e-9)
        fixed = max(t1 - 4096 * per, 0.0)
        nw = int(min(1 << 24, max(4096, (budget_s - fixed) / per)))
        steps, dt = timed(nw, seed_ + 1)
        return nw, steps, dt

    nw, steps, dt = sized(target_s, seed)
    out = {"value": steps / dt, "unit": "steps/s", "cores": cores, "kind": "oracle",
           "sample": f"{nw} {POLICY_NAME[MAIN[name]['policy']]} walkers x {length} (uniform starts) on the same graph after its "
                     f"first update batch; inverse transform over exact u64 prefix sums (rebuilt by every walk call); "
                     f"{steps:.0f} steps in {dt:.1f} s",
           "updated_edges_per_s": len(rec) / t_apply, "update_sample": f"the first batch, {len(rec)} records"}
    if one_thread_s:
        O.set_threads(1)
        try:
            nw1, steps1, dt1 = sized(one_thread_s, seed + 7)
        finally:
            O.set_threads(cores)
        out["one_thread"] = {"value": steps1 / dt1, "unit": "steps/s", "cores": 1,
                             "sample": f"{nw1} walkers, {steps1:.0f} steps in {dt1:.1f} s"}
    del og
    return out


# ------------------------------------------------------------------------------------- arms

def run_reference(args):
    """Reference arm: the CPU oracle (the only reference this paper has), bounded sample per step."""
    import oracle as O

    ws, rank, _ = dist_env()
    if rank != 0:
        return
    wl, batches, _ = main_workload(args.workload, args.steps + args.warmup, args.scale, not args.no_hubs, args.walkers)
    G = wl.graph
    og = O.Graph(G.n, G.row_ptr, G.col, G.w)
    pol = _oracle_policy(O, args.workload)
    nw = min(args.ref_walkers, wl.nwalkers)
    total_steps, total_t = 0.0, 0.0
    for i in range(args.warmup + args.steps):
        st = W.walk_starts(G.n, nw, 1000 + i)
        t0 = time.perf_counter()
        og.apply(batches[i], G.max_bits)
        _, plen = og.walk(st, [pol], 1000 + i)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            total_steps += float((plen.astype(np.int64) - 1).sum())
            total_t += dt
    v = total_steps / total_t
    line = {"impl": "reference", "metric": METRIC_MAIN, "value": v,
            "unit": "steps/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total_t / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32/u64", "data": "synthetic",
            "config": dict(main_config(args, wl), sample=f"{nw} of the {wl.nwalkers} walkers per step (bounded "
                                                          f"sample on host cores), every update of the batch"),
            "cpu_baseline": {"value": v, "unit": "steps/s", "cores": O.num_threads(), "kind": "oracle",
                             "sample": f"per step: one batch of updates applied to the oracle, then {nw} walkers "
                                       f"(cap {MAIN[args.workload]['length']})"},
            "e2e": {"value": v, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _ev(torch):
    return torch.cuda.Event(enable_timing=True)


def _policies(B, name):
    spec = MAIN[name]
    if spec["policy"] == "ppr":
        return [B.policy(B.PPR, spec["length"], spec["ppr_stop"])]
    return [B.policy(B.DEEPWALK, spec["length"])]


def walk_roofline(B, g, torch, paths, plen, walk_ms, pk, pk_src, traffic, nsample=10 ** 6):
    """Algorithmic bytes of a walk launch from the per-step model: the mean model bytes of a step over
    a uniform sample of the launch's steps (each counted from the exported state of the vertex it
    leaves) times the launch's step count; over the launch's CUDA-event time."""
    plen_h = plen.cpu().numpy().view(np.uint32)
    w, t, tot = sample_steps(plen_h, nsample, 12345)
    wi = torch.from_numpy(w).to(paths.device)
    ti = torch.from_numpy(t).to(paths.device)
    src = paths[wi, ti].cpu().numpy().view(np.uint32)
    ids, row = np.unique(src, return_inverse=True)
    exv = g.export_vertices(ids)
    per = expected_bytes_per_vertex(exv)
    bps = float(per[row].mean())
    abytes = bps * tot
    achieved = abytes / (walk_ms / 1e3) / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
            "frac": achieved / pk["hbm_gbs"], "traffic": traffic, "kernel": "k_walk_persistent",
            "peak_source": f"{pk_src} hbm_gbs (copy bandwidth)", "bytes_per_step": bps, "steps_per_launch": tot,
            "model": f"per-step model bytes averaged over {len(w)} uniformly sampled steps of the launch "
                     f"({len(ids)} distinct vertices exported) x the launch's steps"}


def update_roofline(g, rec_dev, rec, upd_ms_mean, pk, stream):
    """The update byte model over one further batch of the stream (the touched vertices exported before
    and after it, outside the timed region) over the mean time of the timed batches."""
    ids = np.unique(rec[:, 0])
    ex0 = g.export_vertices(ids)
    g.apply_updates(rec_dev, stream=stream)
    ex1 = g.export_vertices(ids)
    ub = update_bytes(ex0, ex1, rec, ids=ids)
    ach = ub / (upd_ms_mean / 1e3) / 1e9
    return {"bound": "hbm", "achieved": ach, "peak": pk["hbm_gbs"], "unit": "GB/s", "frac": ach / pk["hbm_gbs"],
            "kernel": "update pipeline (one captured graph per batch)", "bytes_per_update": ub / len(rec),
            "model": "per record, sort, locate, adjacency slot, list-group entries, count lines"}


def run_main(args, name, dev, rank, ws, local, secondary=False):
    """One main-workload run: W warm-up and K timed steps (update batch + walk), rooflines, end to end
    through the C ABI with host buffers; for the headline also streaming, the batch sweep and the
    oracle baseline.  Returns the line's fields."""
    import torch
    import torch.distributed as dist

    import paper_2504_10233_gb300 as B

    spec = MAIN[name]
    nsteps = args.warmup + args.steps
    t_setup = time.perf_counter()
    # after the timed steps: one more batch for the update byte model and one for the end-to-end warm-up
    wl, batches, sweep_rec = main_workload(name, nsteps + 2 + min(args.steps, 3), None if secondary else args.scale,
                                           secondary or not args.no_hubs, None if secondary else args.walkers)
    t_gen = time.perf_counter() - t_setup
    G = wl.graph
    stream = torch.cuda.Stream(device=dev)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    t0 = time.perf_counter()
    g = B.Graph(G.n, t(G.row_ptr), t(G.col), t(G.w), max_bits=G.max_bits)
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    t_create = time.perf_counter() - t0
    nw, L = wl.nwalkers, spec["length"]
    stride = L + 1
    starts = t(W.walk_starts(G.n, nw, wl.walk_seed))
    paths = torch.empty((nw, stride), dtype=torch.int32, device=dev)
    plen = torch.empty(nw, dtype=torch.int32, device=dev)
    pol = _policies(B, name)
    recs = [t(b) for b in batches]
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    mode = B.WALK_PERSISTENT | B.WALK_NO_PAD
    if args.autotune:
        with torch.cuda.stream(stream):
            g.autotune(starts, L, stream=stream)  # every walker: the tuned shape fits the whole launch
    seed0 = replica_seed(wl.walk_seed, rank)

    upd_ms, walk_ms, tot_steps, tot_upd = [], [], 0, 0
    launches0 = None
    sampler = ClockSampler(local)
    if not secondary:
        sampler.start()
        sampler.wait_first()  # the sampler's start-up stays out of the timed region
    for i in range(nsteps):
        timed = i >= args.warmup
        if timed and launches0 is None:
            if ws > 1:
                dist.barrier()
            torch.cuda.synchronize()
            launches0 = g.kernel_launches()
            sampler.mark_start()
            t_wall0 = time.perf_counter()
        flush.fill_(i)  # L2 flush between steps (outside the events)
        torch.cuda.synchronize()
        e0, e1, e2 = _ev(torch), _ev(torch), _ev(torch)
        e0.record(stream)
        g.apply_updates(recs[i], stream=stream)
        e1.record(stream)
        g.walk(starts, pol, seed0 + i, stride, paths, plen, mode=mode, stream=stream)
        e2.record(stream)
        torch.cuda.synchronize()
        if timed:
            upd_ms.append(e0.elapsed_time(e1))
            walk_ms.append(e1.elapsed_time(e2))
            tot_steps += int((plen.to(torch.int64) - 1).sum().item())
            tot_upd += len(batches[i])
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    wall = time.perf_counter() - t_wall0
    sampler.mark_end()
    clocks = sampler.stop() if not secondary else None
    launches = g.kernel_launches() - launches0
    g.check(stream)
    step_ms = [a + b for a, b in zip(upd_ms, walk_ms)]
    t_total = max_over_ranks(sum(step_ms) / 1e3, dev)
    all_steps = sum_over_ranks(float(tot_steps), dev)
    value = all_steps / t_total
    walk_rate = tot_steps / (sum(walk_ms) / 1e3)
    upd_rate = tot_upd / (sum(upd_ms) / 1e3)
    pk, pk_src = peaks()
    traffic = args.traffic if args.traffic is not None else measured_traffic(name)
    roof = walk_roofline(B, g, torch, paths, plen, walk_ms[-1], pk, pk_src, traffic)
    upd_roof = update_roofline(g, recs[nsteps], batches[nsteps], float(np.mean(upd_ms)), pk, stream)

    # end to end through the public API with host buffers (pinned): the batch's records and the walk
    # starts go up, the lengths and the packed paths (bingo_walk_packed: no padding) come back
    h_starts = torch.from_numpy(W.walk_starts(G.n, nw, wl.walk_seed)).pin_memory()
    h_len = torch.empty(nw, dtype=torch.int32).pin_memory()
    h_vert = torch.empty(nw * stride, dtype=torch.int32).pin_memory()
    h_recs = [torch.from_numpy(np.ascontiguousarray(b)).pin_memory() for b in batches[nsteps + 1:]]
    e2e_steps, e2e_t, d2h = 0, 0.0, []
    n_e2e = 0 if args.no_e2e else len(h_recs) - 1
    for i in range(n_e2e + (1 if n_e2e else 0)):  # the first pass is an untimed warm-up (staging buffers)
        flush.fill_(i)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g.apply_updates(h_recs[i], stream=stream)  # host records: H2D inside the call
        tot = g.walk_packed(h_starts, pol, seed0 + 1000 + i, L, h_len, h_vert, stream=stream)
        if i == 0:
            continue
        e2e_t += time.perf_counter() - t0
        e2e_steps += tot - nw
        d2h.append(4 * nw + 4 * tot)
    e2e_t = max_over_ranks(e2e_t, dev)
    e2e = {"value": sum_over_ranks(float(e2e_steps), dev) / e2e_t if e2e_t > 0 else None, "unit": "steps/s",
           "h2d_bytes_per_step": int(h_starts.numel() * 4 + h_recs[0].numel() * 4),
           "d2h_bytes_per_step": int(np.mean(d2h)) if d2h else 0,
           "api": "bingo_apply_updates (host records) + bingo_walk_packed (host starts, lengths and packed paths)"}
    out = {"value": value, "ms_per_step": 1e3 * t_total / args.steps, "walk_steps_per_s": walk_rate,
           "updated_edges_per_s": upd_rate, "update_ms_per_step": float(np.mean(upd_ms)),
           "walk_ms_per_step": float(np.mean(walk_ms)), "wall_s_timed": wall, "clocks": clocks, "e2e": e2e,
           "gpu_launches": int(launches), "roofline": roof, "update_roofline": upd_roof,
           "config": {**main_config(args, wl, name),
                      "l2": f"flushed between steps ({L2_FLUSH_BYTES >> 20} MiB write); state > L2",
                      "setup_s": {"generate": t_gen, "create": t_create},
                      "walk_config": {"lanes_per_walker": g.config().lanes_per_walker,
                                      "warps_per_block": g.config().warps_per_block,
                                      "reg_variant": g.config().reg_variant}}}
    del h_vert, h_len, h_starts, paths, plen
    if not secondary and not args.no_e2e:
        # streaming: records of the same stream applied as batches of one (Section 4.2), device buffers
        srec = t(batches[-1][: args.stream_records])
        torch.cuda.synchronize()
        e0, e1 = _ev(torch), _ev(torch)
        e0.record(stream)
        g.stream_updates(srec, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        one_ms = []
        for j in range(30):  # single-record calls: the latency of one streamed update through the API
            t0 = time.perf_counter()
            g.stream_updates(srec[j: j + 1], stream=stream)
            one_ms.append(1e3 * (time.perf_counter() - t0))
        sps = int(srec.shape[0]) / (e0.elapsed_time(e1) / 1e3)
        out["streaming"] = {"records": int(srec.shape[0]), "updates_per_s": sps,
                            "single_record_call_ms_median": float(np.median(one_ms)),
                            "batched_over_streaming": upd_rate / sps}
    if not secondary and sweep_rec is not None and not args.no_sweep:
        out["batch_sweep"] = update_sweep(g, torch, t, sweep_rec, stream)
    if not secondary:
        out["memory_bytes"] = g.memory_report()
    g.close()
    del recs, starts, g
    torch.cuda.empty_cache()
    if rank == 0 and ws == 1 and not secondary and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(G, batches[0], L, 77, args.cpu_seconds, name=name,
                                           one_thread_s=args.cpu_seconds / 2)
    return out


def update_sweep(g, torch, t, rec, stream):
    """Update batches of 10^3 .. 10^7 records (50/50) applied in place, consecutive slices of the same
    stream; per size the median of the timed batches after one untimed one."""
    off, sweep = 0, []
    for sz in SWEEP_SIZES:
        ms_rep, nf = [], 0
        for rep in range(SWEEP_REPS):
            r = t(rec[off: off + sz])
            off += sz
            torch.cuda.synchronize()
            e0, e1 = _ev(torch), _ev(torch)
            e0.record(stream)
            st = g.apply_updates(r, stream=stream)
            e1.record(stream)
            torch.cuda.synchronize()
            if rep:
                ms_rep.append(e0.elapsed_time(e1))
                nf += st["not_found"]
        ms = float(np.median(ms_rep))
        sweep.append({"batch": sz, "ms": ms, "updated_edges_per_s": sz / (ms / 1e3), "not_found": nf,
                      "timed_batches": len(ms_rep)})
    return sweep


def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_2504_10233_gb300 as B

    ws, rank, local = dist_env()
    if ws > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", init_method="env://")
    dev = torch.device("cuda", local if ws > 1 else 0)
    torch.cuda.set_device(dev)
    B.load()
    main = run_main(args, args.workload, dev, rank, ws, local)
    sec = None
    if args.secondary and args.secondary != args.workload and args.secondary != "none":
        sec = run_main(args, args.secondary, dev, rank, ws, local, secondary=True)
    if rank == 0:
        line = {"metric": METRIC_MAIN,
                "value": main["value"], "unit": "steps/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": main["ms_per_step"], "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "u32/u64", "data": "synthetic", "config": main["config"],
                **{k: v for k, v in main.items() if k not in ("value", "ms_per_step", "config")}}
        if sec is not None:
            line["secondary"] = {"workload": args.secondary, **sec}
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


def _clocks_and_graph(args, name, **mk):
    import torch

    import paper_2504_10233_gb300 as B

    B.load()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    t0 = time.perf_counter()
    wl = W.make_workload(name, **mk)
    t_gen = time.perf_counter() - t0
    G = wl.graph
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    t0 = time.perf_counter()
    g = B.Graph(G.n, t(G.row_ptr), t(G.col), t(G.w), max_bits=G.max_bits)
    torch.cuda.synchronize()
    t_create = time.perf_counter() - t0
    return B, torch, dev, wl, G, g, t, {"generate_s": t_gen, "create_s": t_create}


def run_mixed(args):
    """RMAT-24, 4M walkers in one persistent launch: node2vec (p=2, q=0.5, L=80) and PPR (stop 0.15,
    cap 100) interleaved by walker id, against the same walkers run stepwise (one launch per step) and
    as one launch per policy."""
    B, torch, dev, wl, G, g, t, setup = _clocks_and_graph(args, "c3")
    nw = wl.nwalkers
    stride = 101
    starts = t(W.walk_starts(G.n, nw, wl.walk_seed))
    pids_np = (np.arange(nw) % 2).astype(np.uint8)
    pids = t(pids_np)
    pols = [B.policy(B.NODE2VEC, 80, n2v_pq=(2.0, 0.5)), B.policy(B.PPR, 100, 0.15)]
    paths = torch.empty((nw, stride), dtype=torch.int32, device=dev)
    plen = torch.empty(nw, dtype=torch.int32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    stream = torch.cuda.Stream(device=dev)
    if args.autotune:
        g.autotune(starts[: 1 << 18], 80, stream=stream)
    ev = lambda: torch.cuda.Event(enable_timing=True)
    mode = B.WALK_PERSISTENT | B.WALK_NO_PAD

    def timed_walk(seed, st_, pid_, m_, n_):
        flush.fill_(seed & 0xFF)
        torch.cuda.synchronize()
        e0, e1 = ev(), ev()
        e0.record(stream)
        g.walk(st_, pols, seed, stride, paths[:n_], plen[:n_], policy_ids=pid_, mode=m_, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), int((plen[:n_].to(torch.int64) - 1).sum().item())

    for i in range(args.warmup):
        timed_walk(100 + i, starts, pids, mode, nw)
    sampler = ClockSampler(0)
    sampler.start()
    sampler.wait_first()
    launches0 = g.kernel_launches()
    ms, steps = [], 0
    for i in range(args.steps):
        a, b = timed_walk(200 + i, starts, pids, mode, nw)
        ms.append(a)
        steps += b
    launches = g.kernel_launches() - launches0
    clocks = sampler.stop()
    g.check(stream)
    value = steps / (sum(ms) / 1e3)
    # plain forms on the same walkers
    sw_ms, sw_steps = timed_walk(200, starts, pids, B.WALK_STEPWISE | B.WALK_NO_PAD, nw)
    per_ms, per_steps = 0.0, 0
    for p in (0, 1):
        sel = np.nonzero(pids_np == p)[0]
        a, b = timed_walk(200, t(W.walk_starts(G.n, nw, wl.walk_seed)[sel]), t(pids_np[sel]), mode, len(sel))
        per_ms += a
        per_steps += b
    # roofline model over the last launch, on a uniform sample of its steps: PPR steps and node2vec's
    # first step by the first-order model; later node2vec steps with their rejected candidates and
    # edge-index probes (Eq. node2vec: accept with f(dist)/max f = 1/4, 1/2, 1 at distance 0, 1, 2;
    # the probe is needed when the acceptance draw falls between the distance-1 and -2 thresholds)
    a, b = timed_walk(300, starts, pids, mode, nw)
    abytes, model_note = mixed_walk_bytes(g, torch, paths, plen, pols)
    pk, pk_src = peaks()
    achieved = abytes / (a / 1e3) / 1e9
    cpu = None
    if not args.no_cpu_baseline:
        import oracle as O

        og = O.Graph(G.n, G.row_ptr, G.col, G.w)
        on = 1 << 13
        opol = [O.policy(O.NODE2VEC, 80, 0, [p for p in pols[0].n2v_accept]), O.policy(O.PPR, 100, pols[1].ppr_stop_u32)]
        t0 = time.perf_counter()
        _, ol = og.walk(W.walk_starts(G.n, on, 9), opol, 9, policy_ids=(np.arange(on) % 2).astype(np.uint8))
        dt = time.perf_counter() - t0
        osteps = float((ol.astype(np.int64) - 1).sum())
        cpu = {"value": osteps / dt, "unit": "steps/s", "cores": O.num_threads(), "kind": "oracle",
               "sample": f"{on} walkers (half node2vec, half PPR) on the same graph; {osteps:.0f} steps in {dt:.1f} s"}
    line = {"metric": "sampled walk steps/s, mixed node2vec + PPR in one persistent launch", "value": value,
            "unit": "steps/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": float(np.mean(ms)), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u32/u64", "data": "synthetic",
            "config": {"workload": "RMAT-24 (2^24 vertices, 2^28 edges), fixed-point biases w_fx in [128, 25600); "
                                   "4M walkers: node2vec p=2 q=0.5 L=80 and PPR stop 0.15 cap 100, interleaved",
                       "l2": "flushed between steps; state > L2", "setup": setup,
                       "walk_config": {"lanes_per_walker": g.config().lanes_per_walker,
                                       "warps_per_block": g.config().warps_per_block,
                                       "reg_variant": g.config().reg_variant}},
            "plain_forms": {"stepwise_steps_per_s": sw_steps / (sw_ms / 1e3),
                            "one_launch_per_policy_steps_per_s": per_steps / (per_ms / 1e3),
                            "persistent_over_stepwise": value / (sw_steps / (sw_ms / 1e3))},
            "clocks": clocks, "gpu_launches": int(launches),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
                         "frac": achieved / pk["hbm_gbs"], "traffic": None, "kernel": "k_walk_persistent",
                         "peak_source": f"{pk_src} hbm_gbs", "model": model_note},
            "cpu_baseline": cpu}
    print(json.dumps(line), flush=True)
    g.close()


def mixed_walk_bytes(g, torch, paths, plen, pols, nsample=20000):
    """Model bytes of a launch mixing node2vec (even walker ids) and PPR (odd): the mean model bytes of
    a uniform sample of its steps times its steps."""
    plen_h = plen.cpu().numpy().view(np.uint32)
    w, t, tot = sample_steps(plen_h, nsample, 99)
    P = paths.cpu().numpy().view(np.uint32)
    cur = P[w, t]
    n2v = (w % 2 == 0) & (t >= 1)
    prev = np.where(n2v, P[w, np.maximum(t - 1, 0)], 0)
    ids = np.unique(np.concatenate([cur, prev[n2v]]))
    ex = g.export_vertices(ids)
    fixed, pick = expected_bytes_parts(ex)
    row = np.searchsorted(ids, cur)
    off = np.concatenate([[0], np.cumsum(ex["deg"].astype(np.int64))])
    acc = [int(x) / 2 ** 32 for x in pols[0].n2v_accept]  # accept probability at distance 0, 1, 2
    lo, hi = sorted(acc[1:])
    total = 0.0
    for i in range(len(w)):
        r = row[i]
        if not n2v[i]:
            total += fixed[r] + pick[r] + 4.0
            continue
        rp = np.searchsorted(ids, prev[i])
        dst = ex["dst"][off[r]:off[r + 1]]
        wt = ex["bias"][off[r]:off[r + 1]].astype(np.float64)
        wt /= wt.sum()
        nbr_prev = ex["dst"][off[rp]:off[rp + 1]]
        d1 = np.isin(dst, nbr_prev)
        is_prev = dst == prev[i]
        a = np.where(is_prev, acc[0], np.where(d1, acc[1], acc[2]))
        p_acc = float((wt * a).sum())
        p_probe = float((wt * ~is_prev).sum()) * (hi - lo)
        total += node2vec_step_bytes(fixed[r], pick[r], p_acc, p_probe)
    bps = total / max(len(w), 1)
    return bps * tot, (f"per-step model bytes averaged over {len(w)} sampled steps (node2vec with E[candidates] "
                       f"and edge-index probes): {bps:.1f} B/step")


def run_sweep(args):
    """RMAT-26 + 64 hubs of 10^6 extra out-edges, uniform 31-bit biases: update batches of
    10^3 .. 10^7 (50/50) applied in place, then rounds of 16M PPR walkers (stop 0.15, cap 100)."""
    sizes = [10 ** e for e in range(3, 8)]
    reps = 3  # per size: one untimed batch (capacity growth and graph capture happen there), two timed
    B, torch, dev, wl, G, g, t, setup = _clocks_and_graph(args, "c5", nbatch=1,
                                                          batch=reps * sum(sizes) + 10 ** 6 * (args.steps + args.warmup))
    stream = torch.cuda.Stream(device=dev)
    ev = lambda: torch.cuda.Event(enable_timing=True)
    allrec = wl.batches[0].records()
    off = 0
    sweep = []
    for sz in sizes:
        ms_rep, nf = [], 0
        for rep in range(reps):
            rec = t(allrec[off: off + sz])
            off += sz
            torch.cuda.synchronize()
            e0, e1 = ev(), ev()
            e0.record(stream)
            st = g.apply_updates(rec, stream=stream)
            e1.record(stream)
            torch.cuda.synchronize()
            if rep:
                ms_rep.append(e0.elapsed_time(e1))
                nf += st["not_found"]
        ms = float(np.median(ms_rep))
        sweep.append({"batch": sz, "ms": ms, "updated_edges_per_s": sz / (ms / 1e3), "not_found": nf,
                      "timed_batches": len(ms_rep)})
    nw = wl.nwalkers
    stride = 101
    starts = t(W.walk_starts(G.n, nw, wl.walk_seed))
    paths = torch.empty((nw, stride), dtype=torch.int32, device=dev)
    plen = torch.empty(nw, dtype=torch.int32, device=dev)
    pols = [B.policy(B.PPR, 100, 0.15)]
    mode = B.WALK_PERSISTENT | B.WALK_NO_PAD
    sampler = None
    ms_u, ms_w, steps, nupd = [], [], 0, 0
    for i in range(args.warmup + args.steps):
        rec = t(allrec[off: off + 10 ** 6])
        off += 10 ** 6
        if i == args.warmup:
            sampler = ClockSampler(0)
            sampler.start()
            sampler.wait_first()
            launches0 = g.kernel_launches()
        torch.cuda.synchronize()
        e0, e1, e2 = ev(), ev(), ev()
        e0.record(stream)
        g.apply_updates(rec, stream=stream)
        e1.record(stream)
        g.walk(starts, pols, 500 + i, stride, paths, plen, mode=mode, stream=stream)
        e2.record(stream)
        torch.cuda.synchronize()
        if i >= args.warmup:
            ms_u.append(e0.elapsed_time(e1))
            ms_w.append(e1.elapsed_time(e2))
            steps += int((plen.to(torch.int64) - 1).sum().item())
            nupd += 10 ** 6
    launches = g.kernel_launches() - launches0
    clocks = sampler.stop()
    g.check(stream)
    mem = g.memory_report()
    line = {"metric": "sampled walk steps/s (10^6-update batch + 16M PPR walkers per step); updated edges/s sweep",
            "value": steps / ((sum(ms_u) + sum(ms_w)) / 1e3), "unit": "steps/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": float(np.mean(np.array(ms_u) + np.array(ms_w))),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32/u64", "data": "synthetic",
            "config": {"workload": "RMAT-26 (2^26 vertices, 2^30 edges) + 64 hubs x 10^6 extra out-edges, uniform "
                                   "biases in [1, 2^31); batches 50/50 from the hold-out protocol; 16M PPR walkers",
                       "setup": setup, "memory_bytes": mem},
            "walk_steps_per_s": steps / (sum(ms_w) / 1e3), "updated_edges_per_s": nupd / (sum(ms_u) / 1e3),
            "batch_sweep": sweep, "clocks": clocks, "gpu_launches": int(launches)}
    print(json.dumps(line), flush=True)
    g.close()


def run_serving(args):
    """RMAT-22, uniform 16-bit biases: a Poisson stream of single-edge updates (10^5/s, 70% insert)
    interleaved with Poisson walk requests of 1..10^4 walkers (log-uniform), DeepWalk length 40,
    served by the continuous-batching server; p50/p99 latency per offered request rate, merged
    launches against one launch per request."""
    import ctypes

    B, torch, dev, wl, G, g, t, setup = _clocks_and_graph(args, "c4", nbatch=1, batch=int(1e5 * args.serve_seconds * 8))
    L = B.load()
    ups = np.ascontiguousarray(wl.batches[0].records())
    pol = B.policy(B.DEEPWALK, 40)
    results = []
    uoff = 0
    for merge in (True, False):
        for rate in args.serve_rates:
            rng_u = W.uniform01(200000, 12345 + int(rate), 0)
            gaps = -np.log(1.0 - rng_u) / rate
            arrivals = np.cumsum(gaps)
            arrivals = arrivals[arrivals < args.serve_seconds]
            sizes = np.floor(10 ** (4 * W.uniform01(len(arrivals), 777 + int(rate), 1))).astype(np.int64)
            sizes = np.maximum(sizes, 1)
            nup = int(1e5 * args.serve_seconds)
            up_times = np.arange(nup) / 1e5
            cfg = B.bingo_server_config()
            cfg.flags = 0 if merge else B.SERVER_NO_MERGE
            h = ctypes.c_void_p()
            assert L.bingo_server_create(g.h, ctypes.byref(cfg), ctypes.byref(h)) == 0
            starts_all = W.walk_starts(G.n, int(sizes.sum()) + 1, 4242 + int(rate))
            soff = np.concatenate([[0], np.cumsum(sizes)])
            tickets = []
            done = []

            def collector():
                p = np.zeros((10 ** 4, 41), np.uint32)
                l = np.zeros(10 ** 4, np.uint32)
                ep = ctypes.c_uint64()
                k = 0
                while True:
                    while k >= len(tickets):
                        if done:
                            return
                        time.sleep(0.0002)
                    L.bingo_server_wait(h, tickets[k], 120000, p.ctypes.data, l.ctypes.data, ctypes.byref(ep))
                    k += 1

            th = threading.Thread(target=collector, daemon=True)
            th.start()
            ui = 0
            ri = 0
            t0 = time.perf_counter()
            while ri < len(arrivals) or ui < nup:
                now = time.perf_counter() - t0
                uj = ui
                while uj < nup and up_times[uj] <= now:
                    uj += 1
                if uj > ui:
                    chunk = ups[uoff + ui: uoff + uj]
                    L.bingo_server_submit_updates(h, chunk.ctypes.data, len(chunk), None)
                    ui = uj
                while ri < len(arrivals) and arrivals[ri] <= now:
                    st = starts_all[soff[ri]: soff[ri + 1]]
                    tk = ctypes.c_uint64()
                    L.bingo_server_submit_walk(h, st.ctypes.data, len(st), ctypes.byref(pol), 1000 + ri, ctypes.byref(tk))
                    tickets.append(tk.value)
                    ri += 1
                time.sleep(0.00005)
            L.bingo_server_drain(h, 600000)
            elapsed = time.perf_counter() - t0
            done.append(1)
            th.join(timeout=600)
            stt = B.bingo_server_stats()
            L.bingo_server_stats_get(h, ctypes.byref(stt))
            L.bingo_server_destroy(h)
            uoff += nup
            results.append({"merged": merge, "offered_req_per_s": rate, "requests": int(stt.requests_done),
                            "p50_ms": stt.p50_ms, "p99_ms": stt.p99_ms, "mean_ms": stt.mean_ms,
                            "walk_steps_per_s": stt.steps_done / elapsed, "updates_applied": int(stt.updates_applied),
                            "epochs": int(stt.epochs), "elapsed_s": elapsed})
    g.check()
    mid = [r for r in results if r["merged"] and r["offered_req_per_s"] == args.serve_rates[len(args.serve_rates) // 2]][0]
    line = {"metric": "p99 request latency (ms) under a Poisson request and update stream; walk steps/s served",
            "value": mid["p99_ms"], "unit": "ms", "n_gpus": 1, "steps": len(results), "warmup": 0,
            "ms_per_step": None, "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "u32/u64",
            "data": "synthetic",
            "config": {"workload": "RMAT-22 (2^22 vertices, 2^26 edges), biases U[1, 2^16); updates 10^5/s (70% "
                                   "insert); requests of floor(10^U[0,4]) DeepWalk walkers, L = 40",
                       "offered_req_per_s_for_value": mid["offered_req_per_s"], "setup": setup,
                       "seconds_per_rate": args.serve_seconds},
            "sweep": results}
    print(json.dumps(line), flush=True)
    g.close()


def _timed_walks(torch, B, g, starts, stride, nsteps, warmup, seed0, flush, stream):
    """Median CUDA-event time of `nsteps` DeepWalk launches (after `warmup`), L2 flushed before each."""
    nw = len(starts)
    paths = torch.empty((nw, stride), dtype=torch.int32, device=starts.device)
    plen = torch.empty(nw, dtype=torch.int32, device=starts.device)
    pol = [B.policy(B.DEEPWALK, stride - 1)]
    ms, steps = [], 0
    for i in range(warmup + nsteps):
        flush.fill_(i)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g.walk(starts, pol, seed0 + i, stride, paths, plen, mode=B.WALK_PERSISTENT | B.WALK_NO_PAD, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        if i >= warmup:
            ms.append(e0.elapsed_time(e1))
            steps = int((plen.to(torch.int64) - 1).sum().item())
    g.check(stream)
    return float(np.median(ms)), steps


def _timed_batches(torch, g, recs, warmup, flush, stream):
    ms, conv = [], np.zeros((5, 5), dtype=np.int64)
    for i, r in enumerate(recs):
        flush.fill_(i)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = g.apply_updates(r, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        if i >= warmup:
            ms.append(e0.elapsed_time(e1))
        conv += np.array(st["conversions"])
    return float(np.median(ms)), conv


def run_ablation(args):
    """f1: real-valued biases with lambda (Section 4.3) against the integer graph of their integer
    parts; f2: group adaption (Eq. group) against the all-regular baseline (Section 6.2); f3: radix
    base 4 against base 2 (Appendix).  Same RMAT-20 graph, walkers and batch sizes as the main bench
    workload."""
    import torch

    import paper_2504_10233_gb300 as B

    B.load()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    nb = args.warmup + args.steps
    wl = W.make_workload("c2", nbatch=nb)
    G = wl.graph
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    starts = t(W.walk_starts(G.n, wl.nwalkers, wl.walk_seed))
    stride = wl.length + 1
    sampler = ClockSampler(0)
    if args.workload == "f1":
        lam = 10.0
        rng = np.random.default_rng(31)  # real biases uniform in [0.5, 100), the range of the float workload
        breal = rng.uniform(0.5, 100.0, size=len(G.col)).astype(np.float32)
        real = B.Graph(G.n, t(G.row_ptr), t(G.col), t(breal.view(np.uint32)), bias_format=B.BIAS_F32, lambda_=lam)
        ex = real.export_state()  # integer parts of the real graph, in the same CSR order
        integer = B.Graph(G.n, t(G.row_ptr), t(G.col), t(ex["bias"]), max_bits=32)
        recs_r, recs_i = [], []
        for b in wl.batches:
            r = b.records().copy()
            ins = r[:, 3] != 1
            br = rng.uniform(0.5, 100.0, size=int(ins.sum())).astype(np.float32)
            ri = r.copy()
            r[ins, 2] = br.view(np.uint32)
            ri[ins, 2] = np.floor(lam * br.astype(np.float64)).astype(np.uint32)
            recs_r.append(t(r))
            recs_i.append(t(ri))
        sampler.start()
        sampler.wait_first()
        w_r, steps_r = _timed_walks(torch, B, real, starts, stride, args.steps, args.warmup, 7, flush, stream)
        w_i, steps_i = _timed_walks(torch, B, integer, starts, stride, args.steps, args.warmup, 7, flush, stream)
        u_r, _ = _timed_batches(torch, real, recs_r, args.warmup, flush, stream)
        u_i, _ = _timed_batches(torch, integer, recs_i, args.warmup, flush, stream)
        clocks = sampler.stop()
        mr, mi = real.memory_report(), integer.memory_report()
        state_r = sum(v for k, v in mr.items() if k != "pool_capacity")
        state_i = sum(v for k, v in mi.items() if k != "pool_capacity")
        ex = real.export_state()
        cnt = ex["cnt"].astype(np.float64)
        WI = (cnt[:, :31] * np.exp2(np.arange(31) + 8)).sum(axis=1)
        share = np.where(WI + cnt[:, 31] > 0, cnt[:, 31] / np.maximum(WI + cnt[:, 31], 1), 0)
        line = {"metric": "walk time, real-valued over integer biases (Section 4.3)", "value": w_r / w_i, "unit": "x",
                "higher_is_better": False, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
                "dtype": "u32 integer parts + u8 decimal parts", "data": "synthetic",
                "config": {"workload": "RMAT-20 (2^20 vertices, 2^24 edges), real biases uniform in [0.5, 100), "
                                       "lambda = 10; integer twin: the same graph with biases floor(lambda b); "
                                       "2^20 DeepWalk x 80; batches of 10^5 updates (50/50)",
                           "l2": "flushed before every launch"},
                "walk_ms": {"real": w_r, "integer": w_i},
                "walk_steps_per_s": {"real": steps_r / (w_r / 1e3), "integer": steps_i / (w_i / 1e3)},
                "update_ms_per_batch": {"real": u_r, "integer": u_i},
                "state_bytes": {"real": state_r, "integer": state_i, "ratio": state_r / state_i},
                "decimal_share_mean_over_vertices": float(share[ex["deg"] > 0].mean()),
                "paper_context": "A100: 1.02x time, 1.08x memory (real vs integer biases)",
                "clocks": clocks}
    elif args.workload == "f3":
        w20 = np.minimum(G.w, (1 << 20) - 1).astype(np.uint32)  # base 4 takes biases below 4^10
        recs = []
        for b in wl.batches:
            r = b.records().copy()
            r[:, 2] = np.minimum(r[:, 2], (1 << 20) - 1)
            recs.append(t(r))
        g2 = B.Graph(G.n, t(G.row_ptr), t(G.col), t(w20), max_bits=20)
        g4 = B.Graph(G.n, t(G.row_ptr), t(G.col), t(w20), max_bits=20, radix_base=4)
        sampler.start()
        sampler.wait_first()
        w_2, steps = _timed_walks(torch, B, g2, starts, stride, args.steps, args.warmup, 7, flush, stream)
        w_4, _ = _timed_walks(torch, B, g4, starts, stride, args.steps, args.warmup, 7, flush, stream)
        u_2, _ = _timed_batches(torch, g2, recs, args.warmup, flush, stream)
        u_4, _ = _timed_batches(torch, g4, recs, args.warmup, flush, stream)
        clocks = sampler.stop()
        tot = lambda m: sum(v for k, v in m.items() if k not in ("pool_capacity", "edge_index"))
        m2, m4 = g2.memory_report(), g4.memory_report()
        e2, e4 = g2.export_state(), g4.export_state()
        ne = lambda e: int((e["cnt"] > 0).sum())
        line = {"metric": "radix base 4 over base 2: state memory, walk time, update time (Appendix)",
                "value": tot(m4) / tot(m2), "unit": "x (memory)", "higher_is_better": False,
                "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "dtype": "u32/u64", "data": "synthetic",
                "config": {"workload": "RMAT-20 (2^20 vertices, 2^24 edges), floor(Pareto 1.5) biases clipped below "
                                       "2^20; 2^20 DeepWalk x 80; batches of 10^5 updates (50/50)",
                           "l2": "flushed before every launch"},
                "memory_bytes": {"base2": m2, "base4": m4},
                "nonempty_groups": {"base2": ne(e2), "base4": ne(e4)},
                "member_entries": {"base2": int(e2["sizes"]["list_entries"]), "base4": int(e4["sizes"]["list_entries"])},
                "walk_ms": {"base2": w_2, "base4": w_4}, "walk_steps_per_s_base4": steps / (w_4 / 1e3),
                "update_ms_per_batch": {"base2": u_2, "base4": u_4},
                "paper_context": "not evaluated in the paper (larger bases reduce K; nested structures are hard on GPUs)",
                "clocks": clocks}
    else:
        ga = B.Graph(G.n, t(G.row_ptr), t(G.col), t(G.w), max_bits=G.max_bits)
        mem_ga = ga.memory_report()
        bsg = None
        try:
            bsg = B.Graph(G.n, t(G.row_ptr), t(G.col), t(G.w), max_bits=G.max_bits, all_regular=1)
        except B.BingoError as e:  # the baseline may not fit where group adaption does
            bs_err = str(e)
        recs = [t(b.records()) for b in wl.batches]
        sampler.start()
        sampler.wait_first()
        w_ga, steps = _timed_walks(torch, B, ga, starts, stride, args.steps, args.warmup, 7, flush, stream)
        u_ga, conv = _timed_batches(torch, ga, recs, args.warmup, flush, stream)
        mem_bs = w_bs = u_bs = None
        if bsg is not None:
            mem_bs = bsg.memory_report()
            w_bs, _ = _timed_walks(torch, B, bsg, starts, stride, args.steps, args.warmup, 7, flush, stream)
            u_bs, _ = _timed_batches(torch, bsg, recs, args.warmup, flush, stream)
        # alpha / beta sweep of Eq. group (percent thresholds) on the same graph and batches
        sweep = []
        for al, be in ((20, 10), (40, 10), (60, 10), (80, 10), (100, 10), (40, 0), (40, 5), (40, 20)):
            gs = B.Graph(G.n, t(G.row_ptr), t(G.col), t(G.w), max_bits=G.max_bits, alpha_pct=al, beta_pct=be)
            ms_ = gs.memory_report()
            w_s, _ = _timed_walks(torch, B, gs, starts, stride, 3, 2, 7, flush, stream)
            u_s, _ = _timed_batches(torch, gs, recs[:5], 2, flush, stream)
            kinds = np.bincount(gs.export_state()["kind"].reshape(-1), minlength=5)
            sweep.append({"alpha_pct": al, "beta_pct": be,
                          "state_bytes": sum(v for k, v in ms_.items() if k not in ("pool_capacity", "edge_index")),
                          "walk_ms": w_s, "update_ms_per_batch": u_s,
                          "groups_by_kind": dict(zip(["empty", "dense", "one", "sparse", "regular"],
                                                     [int(x) for x in kinds]))})
            del gs
        grp = lambda m: m["regular_groups"] + m["sparse_groups"]
        tot = lambda m: sum(v for k, v in m.items() if k not in ("pool_capacity", "edge_index"))
        # the group-adaption tuner (bingo_autotune_adaption): its pick with no memory limit, and within the
        # state size of the paper's thresholds (alpha 40, beta 10)
        tuned = {}
        for label, budget in (("no_budget", 0), ("within_paper_default_state", tot(mem_ga))):
            tg = B.Graph.tuned(G.n, t(G.row_ptr), t(G.col), t(G.w), starts, wl.length, state_budget_bytes=budget,
                               max_bits=G.max_bits)
            w_t, _ = _timed_walks(torch, B, tg, starts, stride, 3, 2, 7, flush, stream)
            tuned[label] = {"alpha_pct": tg.cfg.alpha_pct, "beta_pct": tg.cfg.beta_pct,
                            "state_bytes": tot(tg.memory_report()), "walk_ms": w_t}
            tg.close()
        clocks = sampler.stop()
        line = {"metric": "memory of the sampling state, all-regular baseline over group adaption (Section 6.2)",
                "value": (tot(mem_bs) / tot(mem_ga)) if mem_bs else None, "unit": "x", "higher_is_better": True,
                "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "dtype": "u32/u64", "data": "synthetic",
                "config": {"workload": "RMAT-20 (2^20 vertices, 2^24 edges), floor(Pareto 1.5) biases; 2^20 DeepWalk "
                                       "x 80; batches of 10^5 updates (50/50)", "l2": "flushed before every launch"},
                "memory_bytes": {"ga": mem_ga, "bs": mem_bs},
                "group_memory_ratio": (grp(mem_bs) / max(1, grp(mem_ga))) if mem_bs else None,
                "walk_ms": {"ga": w_ga, "bs": w_bs}, "walk_steps_per_s_ga": steps / (w_ga / 1e3),
                "update_ms_per_batch": {"ga": u_ga, "bs": u_bs},
                "ga_conversions_all_batches": conv.tolist(),
                "alpha_beta_sweep": sweep,
                "adaption_autotune": tuned,
                "paper_context": "A100: GA uses 14.6-22.2x less memory than BS and is 1.09x faster overall",
                "clocks": clocks}
        if bsg is None:
            line["bs_unavailable"] = bs_err
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=7)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c5")
    ap.add_argument("--secondary", default="c2", help="a second main workload reported beside the headline (none: off)")
    ap.add_argument("--scale", type=int, default=None, help="smaller RMAT scale of the main workload (profiling)")
    ap.add_argument("--no-sweep", action="store_true", help="skip the update batch-size sweep (profiling)")
    ap.add_argument("--no-hubs", action="store_true", help="leave out the main workload's hub edges (profiling)")
    ap.add_argument("--walkers", type=int, default=None, help="fewer walkers per step than the workload's (profiling)")
    ap.add_argument("--autotune", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end pass (profiling runs)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-walkers", type=int, default=16384)
    ap.add_argument("--traffic", type=float, default=None, help="ncu dram bytes per walk launch, if captured")
    ap.add_argument("--stream-records", type=int, default=20000)
    ap.add_argument("--serve-rates", type=float, nargs="+", default=[100.0, 1000.0, 10000.0])
    ap.add_argument("--serve-seconds", type=float, default=2.0)
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "c3":
        run_mixed(args)
    elif args.workload == "c4":
        run_serving(args)
    elif args.workload == "c5-sweep":
        run_sweep(args)
    elif args.workload in ("f1", "f2", "f3"):
        run_ablation(args)
    elif args.workload in MAIN:
        run_ours(args)
    else:
        raise SystemExit(f"unknown workload {args.workload}")


if __name__ == "__main__":
    main()
