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
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
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


def walk_bytes(per_vertex, paths, plen):
    """Sum of per-step bytes over the recorded walks (steps leave from paths[:, t], t < plen-1)."""
    L = paths.shape[1]
    valid = np.arange(L - 1)[None, :] < (plen.astype(np.int64)[:, None] - 1)
    src = paths[:, :-1][valid].astype(np.int64)
    return float(per_vertex[src].sum())


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


# ------------------------------------------------------------------------------------- CPU baseline

def cpu_baseline(G, batch, length, seed, target_s=15.0):
    """The oracle as it stands, on a bounded sample: the first update batch applied, then as many
    DeepWalk walkers as fit in about target_s seconds (calibrated on a small run)."""
    import oracle as O

    og = O.Graph(G.n, G.row_ptr, G.col, G.w)
    og.apply(batch.records(), G.max_bits)
    pol = O.policy(O.DEEPWALK, length)
    nw = 4096
    st = W.walk_starts(G.n, nw, seed)
    t0 = time.perf_counter()
    _, plen = og.walk(st, [pol], seed)
    dt = time.perf_counter() - t0
    rate = max(float((plen.astype(np.int64) - 1).sum()) / max(dt, 1e-9), 1.0)
    nw = int(min(1 << 22, max(nw, target_s * rate / max(length * 0.5, 1))))
    st = W.walk_starts(G.n, nw, seed + 1)
    t0 = time.perf_counter()
    _, plen = og.walk(st, [pol], seed + 1)
    dt = time.perf_counter() - t0
    steps = float((plen.astype(np.int64) - 1).sum())
    return {"value": steps / dt, "unit": "steps/s", "cores": O.num_threads(), "kind": "oracle",
            "sample": f"{nw} DeepWalk walkers x {length} (uniform starts) on the same graph after its first "
                      f"update batch; inverse-CDF over exact u64 prefix sums; {steps:.0f} steps in {dt:.1f} s"}


# ------------------------------------------------------------------------------------- arms

WORKLOAD_TEXT = {
    "c2": "RMAT-20 (2^20 vertices, 2^24 edges, a=.57 b=.19 c=.19), floor(Pareto 1.5) biases <= 2^20; "
          "per step: 10^5 updates (50/50) then 2^20 DeepWalk walkers x 80",
}


def run_reference(args):
    """Reference arm: the CPU oracle (the only reference this paper has), bounded sample per step."""
    import oracle as O

    ws, rank, _ = dist_env()
    if rank != 0:
        return
    wl = W.make_workload(args.workload, nbatch=args.steps + args.warmup)
    G = wl.graph
    og = O.Graph(G.n, G.row_ptr, G.col, G.w)
    pol = O.policy(O.DEEPWALK, wl.length)
    nw = args.ref_walkers
    total_steps, total_t = 0.0, 0.0
    for i in range(args.warmup + args.steps):
        st = W.walk_starts(G.n, nw, 1000 + i)
        t0 = time.perf_counter()
        og.apply(wl.batches[i].records(), G.max_bits)
        _, plen = og.walk(st, [pol], 1000 + i)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            total_steps += float((plen.astype(np.int64) - 1).sum())
            total_t += dt
    v = total_steps / total_t
    line = {"impl": "reference", "metric": "sampled walk steps/s (update batch + walk per step)", "value": v,
            "unit": "steps/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total_t / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32/u64", "data": "synthetic",
            "config": {"workload": WORKLOAD_TEXT.get(args.workload, args.workload),
                       "sample": f"{nw} walkers per step (bounded sample on host cores)"},
            "cpu_baseline": {"value": v, "unit": "steps/s", "cores": O.num_threads(), "kind": "oracle",
                             "sample": f"per step: one batch of updates applied to the oracle, then {nw} walkers x "
                                       f"{wl.length}"},
            "e2e": {"value": v, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


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
    nsteps = args.warmup + args.steps
    wl = W.make_workload(args.workload, nbatch=nsteps)
    G = wl.graph
    stream = torch.cuda.Stream(device=dev)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    g = B.Graph(G.n, t(G.row_ptr), t(G.col), t(G.w), max_bits=G.max_bits)
    nw = wl.nwalkers
    stride = wl.length + 1
    starts = t(W.walk_starts(G.n, nw, wl.walk_seed))
    paths = torch.empty((nw, stride), dtype=torch.int32, device=dev)
    plen = torch.empty(nw, dtype=torch.int32, device=dev)
    pol = [B.policy(B.DEEPWALK, wl.length)]
    recs = [t(b.records()) for b in wl.batches]
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    mode = B.WALK_PERSISTENT | B.WALK_NO_PAD
    if args.autotune:
        with torch.cuda.stream(stream):
            g.autotune(starts[: min(nw, 1 << 18)], wl.length, stream=stream)
    seed0 = replica_seed(wl.walk_seed, rank)

    ev = lambda: torch.cuda.Event(enable_timing=True)
    upd_ms, walk_ms, tot_steps, tot_upd = [], [], 0, 0
    launches0 = None
    sampler = ClockSampler(local)
    for i in range(nsteps):
        timed = i >= args.warmup
        if timed and launches0 is None:
            if ws > 1:
                dist.barrier()
            torch.cuda.synchronize()
            launches0 = g.kernel_launches()
            sampler.start()
            t_wall0 = time.perf_counter()
        flush.fill_(i)  # L2 flush between steps (outside the events)
        torch.cuda.synchronize()
        e0, e1, e2 = ev(), ev(), ev()
        e0.record(stream)
        st = g.apply_updates(recs[i], stream=stream)
        e1.record(stream)
        g.walk(starts, pol, seed0 + i, stride, paths, plen, mode=mode, stream=stream)
        e2.record(stream)
        torch.cuda.synchronize()
        if timed:
            upd_ms.append(e0.elapsed_time(e1))
            walk_ms.append(e1.elapsed_time(e2))
            tot_steps += int((plen.to(torch.int64) - 1).sum().item())
            tot_upd += len(wl.batches[i])
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    wall = time.perf_counter() - t_wall0
    clocks = sampler.stop()
    launches = g.kernel_launches() - launches0
    g.check(stream)
    step_ms = [a + b for a, b in zip(upd_ms, walk_ms)]
    t_total = max_over_ranks(sum(step_ms) / 1e3, dev)
    all_steps = sum_over_ranks(float(tot_steps), dev)
    value = all_steps / t_total
    walk_rate = tot_steps / (sum(walk_ms) / 1e3)
    upd_rate = tot_upd / (sum(upd_ms) / 1e3)

    # roofline of the walk kernel from the current state and the last timed walk's paths
    ex = g.export_state()
    per_v = expected_bytes_per_vertex(ex)
    p_np = paths.cpu().numpy().view(np.uint32)
    l_np = plen.cpu().numpy().view(np.uint32)
    abytes = walk_bytes(per_v, p_np, l_np)
    pk, pk_src = peaks()
    achieved = abytes / (walk_ms[-1] / 1e3) / 1e9
    roof = {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
            "frac": achieved / pk["hbm_gbs"], "traffic": args.traffic,
            "kernel": "k_walk_persistent", "peak_source": f"{pk_src} hbm_gbs (copy bandwidth)",
            "bytes_per_step": abytes / max(1, int((l_np.astype(np.int64) - 1).sum()))}

    # end to end through the public API with host buffers (pinned), copies inside the timed region
    h_starts = torch.from_numpy(W.walk_starts(G.n, nw, wl.walk_seed)).pin_memory()
    h_paths = torch.empty((nw, stride), dtype=torch.int32).pin_memory()
    h_plen = torch.empty(nw, dtype=torch.int32).pin_memory()
    h_recs = [torch.from_numpy(np.ascontiguousarray(b.records())).pin_memory() for b in wl.batches]
    e2e_steps, e2e_t = 0, 0.0
    for i in range(0 if args.no_e2e else min(args.steps, 3)):
        flush.fill_(i)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g.apply_updates(h_recs[i % len(h_recs)], stream=stream)  # host records: H2D inside the call
        g.walk(h_starts, pol, seed0 + 1000 + i, stride, h_paths, h_plen, mode=mode, stream=stream)
        e2e_t += time.perf_counter() - t0
        e2e_steps += int((h_plen.numpy().astype(np.int64) - 1).sum())
    e2e_t = max_over_ranks(e2e_t, dev)
    e2e = {"value": sum_over_ranks(float(e2e_steps), dev) / e2e_t if e2e_t > 0 else None, "unit": "steps/s",
           "h2d_bytes_per_step": int(h_starts.numel() * 4 + h_recs[0].numel() * 4),
           "d2h_bytes_per_step": int(h_paths.numel() * 4 + h_plen.numel() * 4)}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(G, wl.batches[0], wl.length, 77, args.cpu_seconds)
    if rank == 0:
        line = {"metric": "sampled walk steps/s (update batch + walk per step); updated edges/s; p50/p99 latency "
                          "in the serving bench",
                "value": value, "unit": "steps/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": 1e3 * t_total / args.steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "u32/u64", "data": "synthetic",
                "config": {"workload": WORKLOAD_TEXT.get(args.workload, args.workload), "walkers": nw,
                           "length": wl.length, "updates_per_step": len(wl.batches[0]),
                           "l2": f"flushed between steps ({L2_FLUSH_BYTES >> 20} MiB write); state > L2",
                           "walk_config": {"lanes_per_walker": g.config().lanes_per_walker,
                                           "warps_per_block": g.config().warps_per_block,
                                           "reg_variant": g.config().reg_variant}},
                "updated_edges_per_s": upd_rate, "walk_steps_per_s": walk_rate,
                "update_ms_per_step": float(np.mean(upd_ms)), "walk_ms_per_step": float(np.mean(walk_ms)),
                "wall_s_timed": wall, "clocks": clocks, "e2e": e2e, "gpu_launches": int(launches),
                "roofline": roof, "cpu_baseline": cpu}
        print(json.dumps(line), flush=True)
    g.close()
    if ws > 1:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=7)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c2")
    ap.add_argument("--autotune", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end pass (profiling runs)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-walkers", type=int, default=16384)
    ap.add_argument("--traffic", type=float, default=None, help="ncu dram bytes per walk launch, if captured")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
