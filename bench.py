#!/usr/bin/env python
"""Benchmark of the RNSM merge path: merged vertices/s on one GB300.

Workload: 2 segments x 500,000 vectors, d = 128, SIFT-like integer Gaussian
mixture (1,000 clusters, values 0..255), squared L2, R = 32, L = 64,
alpha = 1.2, FP32.  A step is one rnsm_merge call (expansion, inversion,
pivot selection, pivot and follower searches, source prune, reverse edges)
over both segments, inputs resident in HBM.  The input segment graphs are
built once, untimed, by rnsm_build_segment.

--impl reference times the FP64 CPU oracle instead (host cores, bounded
sample of the same workload).  Under torchrun every rank runs an independent
replica (the merge is not sharded); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from workloads import generators as gen  # noqa: E402

WORKLOAD = "sift-like 2x500k d128 L2 R32 L64 alpha1.2"
METRIC = "merged_vertices_per_s"
UNIT = "vertices/s"
R, L, ALPHA, DIM = 32, 64, 1.2, 128
CPU_SAMPLE = 50_000          # per-segment rows of the oracle's bounded sample
SEARCH_SRC = os.path.join(ROOT, "paper_2602_17099_gb300", "csrc", "search.cu")
PROFILE = os.path.join(ROOT, "profiles", "search_kernel_sift2x500k.txt")


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def init_dist(ws):
    if ws <= 1:
        return None
    import torch.distributed as dist
    os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
    dist.init_process_group("gloo")
    return dist


def barrier(dist):
    if dist is not None:
        dist.barrier()


def whole_job_rate(units_per_rank_step: int, steps: int, world: int, ms_max: float) -> float:
    """Units all ranks processed divided by the slowest rank's time (1/s)."""
    return units_per_rank_step * steps * world / (ms_max / 1000.0)


def allmax(dist, x: float) -> float:
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", gpu_id],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for nm, v in zip(names, f[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------- oracle arm

def oracle_sample(n_per_seg=CPU_SAMPLE):
    """Bounded sample of the workload for the CPU oracle: the same recipe at
    n_per_seg rows per segment; graphs built by the oracle (untimed)."""
    import oracle
    segs, _ = gen.sift_case(n_per_seg=n_per_seg, nq=10)
    gs = [oracle.build_graph(s, R, L, ALPHA) for s in segs]
    return oracle, segs, gs


def oracle_merge_once(oracle, segs, gs):
    t0 = time.perf_counter()
    oracle.rnsm_merge(segs, [g for g, _ in gs], [e for _, e in gs],
                      oracle.pair_plan([len(s) for s in segs]), R, L, ALPHA)
    return time.perf_counter() - t0


def cpu_baseline():
    oracle, segs, gs = oracle_sample()
    t = oracle_merge_once(oracle, segs, gs)
    n = sum(len(s) for s in segs)
    return {"value": n / t, "unit": UNIT, "cores": oracle.max_threads(), "kind": "oracle",
            "sample": f"2 x {CPU_SAMPLE} rows of the same SIFT-like recipe, one merge, "
                      f"{t:.2f} s (FP64 C oracle, OpenMP)"}


def run_reference(args, ws, rank):
    if rank != 0:
        return 0
    oracle, segs, gs = oracle_sample()
    n = sum(len(s) for s in segs)
    for _ in range(args.warmup):
        oracle_merge_once(oracle, segs, gs)
    total = 0.0
    for _ in range(args.steps):
        total += oracle_merge_once(oracle, segs, gs)
    value = n * args.steps / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000 * total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample_rows_per_segment": CPU_SAMPLE},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.max_threads(),
                             "kind": "oracle",
                             "sample": f"2 x {CPU_SAMPLE} rows per step (FP64 C oracle)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------- our arm

def search_profile_traffic():
    """Per-launch DRAM bytes of the search kernel from the committed ncu
    summary, if it was taken on the current kernel source."""
    try:
        with open(PROFILE) as f:
            txt = f.read()
        with open(SEARCH_SRC, "rb") as f:
            h = hashlib.sha256(f.read()).hexdigest()[:16]
    except OSError:
        return None
    meta = {}
    for line in txt.splitlines():
        if ":" in line:
            k, v = line.split(":", 1)
            meta[k.strip()] = v.strip()
    if meta.get("search.cu sha256[:16]") != h:
        return None
    try:
        return float(meta["dram bytes per full-size launch"])
    except (KeyError, ValueError):
        return None


def recall_at_10(rn, torch, Xd, adj, entry, Q, ef=64):
    """Tie-tolerant Recall@10 of the merged graph (evaluation only)."""
    Qd = torch.from_numpy(Q).cuda()
    seeds = torch.full((len(Q), 1), entry, dtype=torch.int32, device="cuda")
    ids, _, _ = rn.search(Xd, adj, Qd, seeds, ef, 10)
    # exact 10-NN distances: integer data, exact in FP32
    d10 = []
    for b in range(0, len(Q), 256):
        q = Qd[b:b + 256]
        dd = (q * q).sum(1, keepdim=True) + (Xd * Xd).sum(1)[None] - 2.0 * (q @ Xd.T)
        d10.append(torch.topk(dd, 10, largest=False).values[:, 9])
    d10 = torch.cat(d10)
    got = Xd[ids.clamp(min=0).long()]
    dg = ((got - Qd[:, None, :]) ** 2).sum(-1)
    hit = ((dg <= d10[:, None]) & (ids >= 0)).sum().item()
    return hit / (10 * len(Q))


def run_ours(args, ws, rank, local):
    import torch

    from paper_2602_17099_gb300 import build as pkg_build
    from paper_2602_17099_gb300 import rnsm as rn

    dist = init_dist(ws)
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device (there is no CPU path)")
    torch.cuda.set_device(local)
    if rank == 0 or ws == 1:
        pkg_build.build()
    barrier(dist)
    rn.lib()

    n_per = args.n_per_seg
    segs, Q = gen.sift_case(n_per_seg=n_per, nq=args.recall_queries)
    N = sum(len(s) for s in segs)
    vd = [torch.from_numpy(s).cuda() for s in segs]
    t0 = time.perf_counter()
    graphs = [rn.build_segment(v, R, L, ALPHA) for v in vd]
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    tsegs = [(v, g, e) for v, (g, e) in zip(vd, graphs)]
    p = rn.params(R, L, ALPHA)
    out = torch.empty((N, R), dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()

    for _ in range(args.warmup):
        rn.merge(tsegs, p, out=out)
    torch.cuda.synchronize()

    gpu_id = torch.cuda.get_device_properties(local).uuid
    gpu_id = f"GPU-{gpu_id}" if not str(gpu_id).startswith("GPU-") else str(gpu_id)
    sampler = ClockSampler(gpu_id)
    time.sleep(0.5)
    barrier(dist)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stats = []
    ev0.record(stream)
    for _ in range(args.steps):
        torch.cuda.nvtx.range_push("rnsm_merge")
        _, st = rn.merge(tsegs, p, out=out)
        torch.cuda.nvtx.range_pop()
        stats.append(st)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(dist)
    clocks = sampler.stop()
    ms = ev0.elapsed_time(ev1)
    ms_max = allmax(dist, ms)
    value = whole_job_rate(N, args.steps, ws, ms_max)

    # roofline of the search kernel (S1, S4, S5 launches), from the
    # library's CUDA events on the launching stream and its NDC counters
    s_bytes = s_ms = 0.0
    launches = 0
    for st in stats:
        for i, ph in ((0, 1), (1, 4), (2, 5)):
            s_bytes += (st["search_ndc"][i] * DIM * 4 + st["search_exp"][i] * R * 4 +
                        st["search_queries"][i] * DIM * 4)
            s_ms += st["phase_ms"][ph]
        launches += st["launches"]
    n_search_launches = 3 * len(stats)
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except OSError:
        pass
    peak = float(peaks.get("hbm_gbs", 6800.0))
    achieved = (s_bytes / n_search_launches) / (s_ms / n_search_launches / 1000.0) / 1e9
    traffic = search_profile_traffic()
    roofline = {"bound": "hbm", "kernel": "search_kernel (S1+S4+S5 launches)",
                "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "peak_source": "measured" if "hbm_gbs" in peaks else "fallback",
                "traffic": traffic,
                "algorithmic_bytes_per_launch": s_bytes / n_search_launches,
                "avg_launch_ms": s_ms / n_search_launches}
    phases = ["validate_init", "S1_expand", "S2_invert", "S3_pivots_host", "S4_pivot_search",
              "S5_follower_search", "S6_source_prune", "S7_reverse_edges"]
    phase_ms = {nm: sum(st["phase_ms"][i] for st in stats) / len(stats)
                for i, nm in enumerate(phases)}

    # precision pattern: the same merge with BF16 / FP8 prune tiles (tensor
    # cores + FP32 re-decisions); their graphs must equal the FP32 graph
    modes = {}
    ref_out = out.clone()
    for name, prec in (("bf16", rn.BF16), ("fp8", rn.FP8)):
        pq = rn.params(R, L, ALPHA, prec=prec)
        oq = torch.empty_like(out)
        for _ in range(2):
            rn.merge(tsegs, pq, out=oq)
        torch.cuda.synchronize()
        q0, q1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        qs = []
        nq = max(3, args.steps // 2)
        q0.record(stream)
        for _ in range(nq):
            _, st = rn.merge(tsegs, pq, out=oq)
            qs.append(st)
        q1.record(stream)
        torch.cuda.synchronize()
        qms = q0.elapsed_time(q1) / nq
        modes[name] = {"ms_per_step": qms, "value": N / (qms / 1000.0), "unit": UNIT,
                       "identical_to_fp32": bool(torch.equal(oq, ref_out)),
                       "rechecks_per_step": qs[-1]["rechecks"],
                       "prune_ms": round(sum(st["phase_ms"][6] + st["phase_ms"][7]
                                             for st in qs) / nq, 3)}
    modes["fp32"] = {"ms_per_step": ms_max / args.steps,
                     "prune_ms": round(phase_ms["S6_source_prune"] + phase_ms["S7_reverse_edges"], 3)}

    # end to end through the public API with host buffers
    pin_v = [s_.cpu().pin_memory() for s_ in vd]
    pin_g = [g.cpu().pin_memory() for g, _ in graphs]
    pin_out = torch.empty((N, R), dtype=torch.int32).pin_memory()
    dv = [torch.empty_like(v) for v in vd]
    dg = [torch.empty_like(g) for g, _ in graphs]
    h2d = sum(t.numel() * t.element_size() for t in pin_v + pin_g)
    d2h = pin_out.numel() * pin_out.element_size()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(dist)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        for a, b in zip(dv, pin_v):
            a.copy_(b, non_blocking=True)
        for a, b in zip(dg, pin_g):
            a.copy_(b, non_blocking=True)
        rn.merge([(v, g, e) for v, g, (_, e) in zip(dv, dg, graphs)], p, out=out)
        pin_out.copy_(out, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = allmax(dist, e0.elapsed_time(e1))
    e2e = {"value": whole_job_rate(N, args.steps, ws, e2e_ms), "unit": UNIT,
           "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}

    rec = None
    if rank == 0 and args.recall_queries > 0:
        Xd = torch.cat(vd)
        big = 0 if len(segs[0]) >= len(segs[1]) else 1
        entry = graphs[big][1] + (0 if big == 0 else len(segs[0]))
        rec = {"ef": 64, "queries": args.recall_queries,
               "value": recall_at_10(rn, torch, Xd, out, entry, Q)}

    base = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        base = cpu_baseline()

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic",
                "config": {"workload": WORKLOAD, "segments": [len(s) for s in segs],
                           "dim": DIM, "R": R, "L": L, "alpha": ALPHA, "precision": "fp32",
                           "parallelism": "replicas" if ws > 1 else "single",
                           "l2": "inputs larger than L2 (512 MB of vectors)",
                           "input_graph_build_s": round(build_s, 3),
                           "phase_ms": {k: round(v, 3) for k, v in phase_ms.items()},
                           "recall_at_10": rec,
                           "pivots": stats[-1]["pivots"], "followers": stats[-1]["followers"],
                           "ndc_per_step": stats[-1]["ndc"]},
                "clocks": clocks, "e2e": e2e, "gpu_launches": int(launches),
                "precision_modes": modes,
                "roofline": roofline, "cpu_baseline": base}
        print(json.dumps(line), flush=True)
    barrier(dist)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n-per-seg", type=int, default=500_000)
    ap.add_argument("--recall-queries", type=int, default=1000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    ws, rank, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, ws, rank)
    return run_ours(args, ws, rank, local)


if __name__ == "__main__":
    sys.exit(main())
