#!/usr/bin/env python
"""Benchmark of the RNSM merge path: merged vertices/s on one GB300.

Default workload: 2 segments x 500,000 vectors, d = 128, SIFT-like integer Gaussian
mixture (1,000 clusters, values 0..255), squared L2, R = 32, L = 64,
alpha = 1.2, FP32.  A step is one rnsm_merge call (expansion, inversion,
pivot selection, pivot and follower searches, source prune, reverse edges)
over both segments, inputs resident in HBM.  The input segment graphs are
built once, untimed, by rnsm_build_segment.

Other workloads (--workload): deep10x2m, ten uneven DEEP-like segments
(2M rows, d = 96, cluster partition) merged along a MOS plan that is computed
inside every step; embed4x250k, four 250k-row embedding-like segments
(d = 768, inner product, R = 64, L = 128) along a MOS plan, where the BF16 /
FP8 prune tiles matter most.  --scale shrinks a workload for quick runs.

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

METRIC = "merged_vertices_per_s"
UNIT = "vertices/s"
SEARCH_SRC = [os.path.join(ROOT, "paper_2602_17099_gb300", "csrc", f)
              for f in ("search_impl.cuh", "search.cu", "search_jobs.cu")]
PROFILE = os.path.join(ROOT, "profiles", "search_kernel_sift2x500k.txt")
PRUNE_SRC = [os.path.join(ROOT, "paper_2602_17099_gb300", "csrc", f)
             for f in ("prune.cu", "common.cuh")]
L2_PROFILE = os.path.join(ROOT, "profiles", "search_kernel_s5_sift2x200k.md")
# the FP32 prune kernels of pools <= 64, by the variant number the library
# reports (stats prune_kernel): their kernel name and committed ncu summaries
# (full-size DRAM traffic, small-case FMA-pipe activity)
PRUNE_KERNELS = {
    0: ("prune_small_kernel", "prune_small_kernel_sift2x500k.txt", "prune_small_kernel_sift2x200k.md"),
    3: ("prune_walk_kernel", "prune_walk_kernel_sift2x500k.txt", "prune_walk_kernel_sift2x200k.md"),
}
PRUNE_DEFAULT_VARIANT = 3
L2_METRIC, IP_METRIC = 0, 1


class Workload:
    """One merge workload: segments, queries, parameters and the host plan.

    ``make(scale, nq)`` returns (segments [list of float32 arrays], queries);
    ``oracle_scale`` sizes the CPU oracle's bounded sample: the same recipe
    at that fraction of the full size, with its own plan."""

    def __init__(self, name, desc, dim, R, L, alpha, metric, make, multi, modes, oracle_scale):
        self.name, self.desc, self.dim = name, desc, dim
        self.R, self.L, self.alpha, self.metric = R, L, alpha, metric
        self.make, self.multi, self.modes, self.oracle_scale = make, multi, modes, oracle_scale


def _sift(scale, nq, n_per_seg=None):
    n = n_per_seg if n_per_seg else max(2000, int(500_000 * scale))
    return gen.sift_case(n_per_seg=n, nq=nq)


def _deep(scale, nq):
    total = max(20_000, int(2_000_000 * scale))
    sizes = gen.lognormal_sizes(10, total, max(1000, int(50_000 * scale)),
                                max(4000, int(400_000 * scale)), seed=5)
    X, comp, means = gen.deep_like(total + nq, 5, return_components=True)
    parts = gen.cluster_partition(comp[:total], means, sizes, seed=1005)
    return [X[p_].copy() for p_ in parts], X[total:].copy()


def _embed(scale, nq):
    n = max(2000, int(250_000 * scale))
    X = gen.embed_like(4 * n + nq, 7)
    parts = gen.random_partition(4 * n, 4, 1007)
    return [X[p_].copy() for p_ in parts], X[4 * n:].copy()


def _deep50(scale, nq):
    """50 DEEP-like segments, 100M rows at full size, drawn on the GPU (38 GB)."""
    import torch
    total = max(50_000, int(100_000_000 * scale))
    sizes = gen.lognormal_sizes(50, total, max(1000, int(500_000 * scale)),
                                max(4000, int(5_000_000 * scale)), seed=9)
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    return gen.deep_like_gpu_segments(total, nq, 9, sizes, 1009, device=dev)


def _incremental(scale, nq):
    """10 partitions of a DEEP-like stream in arrival order (1M rows each at full
    size), drawn on the GPU; merged one at a time into a growing index."""
    import torch
    n_part = max(20_000, int(1_000_000 * scale))
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    return gen.deep_like_gpu_segments(10 * n_part, nq, 11, [n_part] * 10, 0, device=dev,
                                      stream=True, return_all=True)


WORKLOADS = {
    "sift2x500k": Workload("sift2x500k", "sift-like 2x500k d128 L2 R32 L64 alpha1.2", 128, 32, 64,
                           1.2, L2_METRIC, _sift, False, ("bf16", "fp8"), 1.0),
    "deep10x2m": Workload("deep10x2m", "deep-like 10 segments (lognormal 50k-400k, 2M total, "
                          "cluster partition) d96 L2 R32 L64 alpha1.2, MOS plan", 96, 32, 64,
                          1.2, L2_METRIC, _deep, True, ("bf16", "fp8"), 0.02),
    "embed4x250k": Workload("embed4x250k", "embedding-like 4x250k d768 IP R64 L128 alpha1.2, "
                            "MOS plan", 768, 64, 128, 1.2, IP_METRIC, _embed, True,
                            ("bf16", "fp8"), 0.01),
    "deep50x100m": Workload("deep50x100m", "deep-like 50 segments (lognormal 0.5M-5M, 100M total, "
                            "cluster partition, drawn on the GPU) d96 L2 R32 L64 alpha1.2, MOS plan",
                            96, 32, 64, 1.2, L2_METRIC, _deep50, True, ("bf16",), 0.01),
    "incr10x1m": Workload("incr10x1m", "deep-like stream d96 L2 R32 L64 alpha1.2: 10 partitions of "
                          "1M in arrival order, each merged into the growing index (9 merges)",
                          96, 32, 64, 1.2, L2_METRIC, _incremental, False, ("bf16",), 0.0),
}


def to_host(x):
    """numpy view of a workload array (device tensors are copied to the host)."""
    return x if isinstance(x, np.ndarray) else x.cpu().numpy()


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

def centroids_of(segs):
    if isinstance(segs[0], np.ndarray):
        return np.stack([s_.mean(axis=0, dtype=np.float64) for s_ in segs]).astype(np.float32)
    return np.stack([s_.double().mean(0).cpu().numpy() for s_ in segs]).astype(np.float32)


def host_plan(W, segs, planner):
    """The merge plan: the single-pair default for two segments, else MOS
    (Algorithm 3) over the segment sizes and centroids."""
    if not W.multi:
        return None
    return planner([len(s_) for s_ in segs], centroids_of(segs))


def oracle_sample(W, args, nq=10):
    """Bounded sample of the workload for the CPU oracle: the same recipe at
    ``W.oracle_scale`` of the full size (and nq queries of the same draw),
    graphs built by the oracle (untimed)."""
    import oracle
    if W.name == "sift2x500k" and args.n_per_seg:
        segs, Q = _sift(1.0, nq, n_per_seg=args.n_per_seg)
    else:
        segs, Q = W.make(W.oracle_scale * args.scale, nq)
    segs = [to_host(s_) for s_ in segs]
    gs = [oracle.build_graph(s_, W.R, W.L, W.alpha, metric=W.metric) for s_ in segs]
    return oracle, segs, gs, to_host(Q)


def sample_plan(W, oracle, segs):
    plan = host_plan(W, segs, lambda sz, c: oracle.mos_plan(sz, c))
    if plan is None:
        plan = oracle.pair_plan([len(s_) for s_ in segs])
    return [(a, b) for a, b, *_ in plan]


def oracle_merge_once(W, oracle, segs, gs, keep=None):
    t0 = time.perf_counter()
    plan = sample_plan(W, oracle, segs)
    merged, _ = oracle.rnsm_merge(segs, [g for g, _ in gs], [e for _, e in gs], plan, W.R, W.L,
                                  W.alpha, metric=W.metric)
    if keep is not None:
        keep["merged"] = merged
    return time.perf_counter() - t0


def recall_parity(W, oracle, segs, gs, Q, merged_oracle, rn, torch, efs=(10, 16, 64)):
    """Recall@10 of the oracle-merged and the GPU-merged graph of the same sample
    (same input graphs, same plan), both searched by the oracle's Algorithm 1
    from the largest segment's entry, against the FP64 brute force, at several
    search efforts (small ones keep recall below 1, where the 0.005 tolerance
    means something)."""
    plan = sample_plan(W, oracle, segs)
    tsegs = [(torch.from_numpy(s_).cuda(), torch.from_numpy(g).cuda(), e) for s_, (g, e) in zip(segs, gs)]
    merged_gpu, _ = rn.merge(tsegs, rn.params(W.R, W.L, W.alpha, metric=W.metric),
                             plan=[(a, b, 0.0) for a, b in plan])
    merged_gpu = merged_gpu.cpu().numpy()
    X = np.concatenate(segs)
    sizes = [len(s_) for s_ in segs]
    big = int(np.argmax(sizes))
    entry = gs[big][1] + sum(sizes[:big])
    _, gd = oracle.bruteforce_knn(X, Q, 10, metric=W.metric)
    seeds = np.full((len(Q), 1), entry, np.int32)
    out = {"queries": len(Q), "ef": list(efs),
           "identical_rows": float((merged_gpu == merged_oracle).all(axis=1).mean()),
           "differing_rows": int((merged_gpu != merged_oracle).any(axis=1).sum())}
    for name, adj in (("oracle_merged", merged_oracle), ("gpu_merged", merged_gpu)):
        out[name] = [oracle.recall_at_k(oracle.beam_search(X, adj, Q, seeds, ef, 10,
                                                           metric=W.metric)[0],
                                        X, gd, Q, metric=W.metric) for ef in efs]
    out["max_abs_diff"] = max(abs(a - b) for a, b in zip(out["oracle_merged"], out["gpu_merged"]))
    out["within_0.005"] = out["max_abs_diff"] <= 0.005
    return out


def sample_desc(W, segs):
    what = ("the workload itself" if W.oracle_scale == 1.0 else
            f"the same recipe at {W.oracle_scale:g} of the workload's size")
    return (f"{what}: {len(segs)} segments, {sum(len(s_) for s_ in segs)} rows, input graphs "
            f"built by the oracle (untimed), FP64 C oracle with OpenMP")


def cpu_baseline(W, args, min_s=10.0, max_runs=40, rn=None, torch=None):
    """The oracle's merge on the bounded sample (the SIFT-like default: the full
    2 x 500k workload), repeated until about min_s of CPU time has been
    measured.  With the library at hand, also the recall parity of the two
    merged graphs on 1,000 queries."""
    oracle, segs, gs, Q = oracle_sample(W, args, nq=1000)
    n = sum(len(s_) for s_ in segs)
    total, runs, keep = 0.0, 0, {}
    while runs < max_runs and (runs == 0 or total < min_s):
        total += oracle_merge_once(W, oracle, segs, gs, keep)
        runs += 1
    out = {"value": n * runs / total, "unit": UNIT, "cores": oracle.max_threads(),
           "kind": "oracle",
           "sample": sample_desc(W, segs) + f", {runs} merges in {total:.2f} s"}
    if rn is not None:
        out["recall_parity"] = recall_parity(W, oracle, segs, gs, Q, keep["merged"], rn, torch)
    return out


def run_reference(args, ws, rank):
    if rank != 0:
        return 0
    W = WORKLOADS[args.workload]
    oracle, segs, gs, _ = oracle_sample(W, args)
    n = sum(len(s_) for s_ in segs)
    for _ in range(args.warmup):
        oracle_merge_once(W, oracle, segs, gs)
    total = 0.0
    for _ in range(args.steps):
        total += oracle_merge_once(W, oracle, segs, gs)
    value = n * args.steps / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000 * total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": W.desc, "sample_segments": [len(s_) for s_ in segs]},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.max_threads(),
                             "kind": "oracle", "sample": sample_desc(W, segs) + " per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------- our arm

def profile_traffic(path, sources, hash_key, bytes_key):
    """Per-launch DRAM bytes from a committed ncu summary, if it was taken on
    the current kernel sources (their sha256 prefix is recorded beside it)."""
    try:
        with open(path) as f:
            txt = f.read()
        hs = hashlib.sha256()
        for src in sources:
            with open(src, "rb") as f:
                hs.update(f.read())
        h = hs.hexdigest()[:16]
    except OSError:
        return None
    meta = {}
    for line in txt.splitlines():
        for key in (hash_key, bytes_key):
            if line.startswith(key + ":"):
                meta[key] = line[len(key) + 1:].strip()
    if meta.get(hash_key) != h:
        return None
    try:
        return float(meta[bytes_key])
    except (KeyError, ValueError):
        return None


def search_profile_traffic():
    return profile_traffic(PROFILE, SEARCH_SRC, "search sources sha256[:16]",
                           "dram bytes per launch (mean of S1, S4, S5)")


def _prune_profile(variant, k):
    v = PRUNE_KERNELS.get(variant)
    return os.path.join(ROOT, "profiles", v[k]) if v else None


def prune_profile_traffic(variant=PRUNE_DEFAULT_VARIANT):
    path = _prune_profile(variant, 1)
    return path and profile_traffic(path, PRUNE_SRC, "prune sources sha256[:16]",
                                    "dram bytes per S6 launch")


def prune_profile_fma(variant=PRUNE_DEFAULT_VARIANT):
    """FMA-pipe activity (percent of peak) of an FP32 small-pool prune kernel,
    from the committed small-case ncu capture of the current sources."""
    path = _prune_profile(variant, 2)
    return path and profile_traffic(path, PRUNE_SRC, "prune sources sha256[:16]",
                                    "fma pipe active pct (S6)")


def search_profile_l2():
    """L2 throughput of the search kernel (percent of its peak) and its L2 hit
    rate, from the committed small-case ncu capture of the current sources."""
    out = {}
    for key in ("l2 throughput pct (S5)", "l2 hit rate pct (S5)"):
        v = profile_traffic(L2_PROFILE, SEARCH_SRC, "search sources sha256[:16]", key)
        if v is not None:
            out[key.replace(" (S5)", "").replace(" ", "_")] = v
    if out:
        out["source"] = os.path.relpath(L2_PROFILE, ROOT)
    return out or None


def recall_at_10(rn, torch, W, Xd, adj, entry, Q, ef=64, chunk_rows=1 << 22, qb=64, gt=None):
    """Tie-tolerant Recall@10 of the merged graph (evaluation only): a returned
    id counts if its FP64 distance is within the true 10th-NN distance.  The
    true neighbours come from a chunked FP32 scan (top 32 per query) re-ranked
    in FP64 (``gt``: the 10th-NN distances of an earlier call, reused).
    entry: one global id, or a list (every query seeded with all).  ``ef`` may
    be a list: the recall at each."""
    Qd = Q if torch.is_tensor(Q) else torch.from_numpy(Q)
    Qd = Qd.cuda()
    nq = Qd.shape[0]
    ent = torch.tensor(entry if isinstance(entry, (list, tuple)) else [entry], dtype=torch.int32,
                       device="cuda")
    seeds = ent[None, :].expand(nq, ent.numel()).contiguous()

    def native(rows64, q64):
        if W.metric == L2_METRIC:
            return ((rows64 - q64[:, None, :]) ** 2).sum(-1)
        return 1.0 - (rows64 * q64[:, None, :]).sum(-1)

    d10 = gt if gt is not None else true_d10(torch, W, Xd, Qd, native, chunk_rows, qb)
    efs = ef if isinstance(ef, (list, tuple)) else [ef]
    res = []
    for e in efs:
        ids, _, _ = rn.search(Xd, adj, Qd, seeds, e, 10, metric=W.metric)
        hit = 0
        for b in range(0, nq, qb):
            q64 = Qd[b:b + qb].double()
            got = ids[b:b + qb]
            ex = native(Xd[got.clamp(min=0).long()].double(), q64)
            dk = d10[b:b + qb]
            tol = 1e-9 * dk.abs()[:, None] + 1e-12
            hit += ((ex <= dk[:, None] + tol) & (got >= 0)).sum().item()
        res.append(hit / (10 * nq))
    return res if isinstance(ef, (list, tuple)) else res[0]


def true_d10(torch, W, Xd, Qd, native, chunk_rows=1 << 22, qb=64):
    """FP64 10th-NN distance of every query: a chunked FP32 scan keeps the best 32
    candidates of each query, re-ranked in FP64."""
    out = []
    for b in range(0, Qd.shape[0], qb):
        q = Qd[b:b + qb]
        best_d = best_i = None
        for c0 in range(0, Xd.shape[0], chunk_rows):
            Xc = Xd[c0:c0 + chunk_rows]
            if W.metric == L2_METRIC:
                approx = (q * q).sum(1, keepdim=True) + (Xc * Xc).sum(1)[None] - 2.0 * (q @ Xc.T)
            else:
                approx = 1.0 - q @ Xc.T
            dv, iv = torch.topk(approx, min(32, Xc.shape[0]), largest=False)
            iv = iv + c0
            if best_d is not None:
                dv, iv = torch.cat([best_d, dv], 1), torch.cat([best_i, iv], 1)
            sel = torch.topk(dv, min(32, dv.shape[1]), largest=False).indices
            best_d, best_i = torch.gather(dv, 1, sel), torch.gather(iv, 1, sel)
        out.append(torch.sort(native(Xd[best_i].double(), q.double()), dim=1).values[:, 9])
    return torch.cat(out)


def concat_rows(torch, vd):
    """The segments as one [N, d] table: a view when they already sit back to
    back in one allocation (device-drawn workloads), else a copy."""
    d = vd[0].shape[1]
    st = vd[0].untyped_storage()
    p, off = vd[0].data_ptr(), 0
    for v in vd:
        if (v.untyped_storage().data_ptr() != st.data_ptr() or v.data_ptr() != p + off * d * 4
                or not v.is_contiguous()):
            return torch.cat(vd)   # separate allocations (even when adjacent)
        off += v.shape[0]
    return torch.empty(0, dtype=vd[0].dtype, device=vd[0].device).set_(
        st, vd[0].storage_offset(), (off, d), (d, 1))


def e2e_room(torch, in_bytes, out_bytes):
    """None if host and device hold a pinned copy of the inputs and outputs and a
    second device copy of the inputs with room to spare, else the reason."""
    avail = None
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    avail = int(line.split()[1]) * 1024
    except OSError:
        pass
    need_host = in_bytes + out_bytes
    if avail is not None and avail < 2 * need_host + (16 << 30):
        return f"host memory: {avail >> 30} GiB available, {need_host >> 30} GiB to pin"
    free, _ = torch.cuda.mem_get_info()
    if free < 1.1 * in_bytes + (4 << 30):
        return f"device memory: {free >> 30} GiB free, {in_bytes >> 30} GiB of inputs to copy"
    return None


def progress(msg):
    """Progress on stderr (the JSON line stays alone on stdout)."""
    print(f"[bench {time.strftime('%H:%M:%S')}] {msg}", file=sys.stderr, flush=True)


def run_ours(args, ws, rank, local):
    import torch

    from paper_2602_17099_gb300 import build as pkg_build
    from paper_2602_17099_gb300 import rnsm as rn

    W = WORKLOADS[args.workload]
    dist = init_dist(ws)
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device (there is no CPU path)")
    torch.cuda.set_device(local)
    if rank == 0 or ws == 1:
        pkg_build.build()
    barrier(dist)
    rn.lib()

    if W.name == "sift2x500k":
        segs, Q = _sift(args.scale, args.recall_queries, n_per_seg=args.n_per_seg)
    else:
        segs, Q = W.make(args.scale, args.recall_queries)
    N = sum(len(s_) for s_ in segs)
    cen = centroids_of(segs)
    vd = [s_ if torch.is_tensor(s_) else torch.from_numpy(s_).cuda() for s_ in segs]
    huge = N > 20_000_000   # tens of GB: fewer repetitions of the extra measurements
    progress(f"{W.name}: {len(vd)} segments, {N} rows on the device")
    t0 = time.perf_counter()
    graphs = [rn.build_segment(v, W.R, W.L, W.alpha, metric=W.metric) for v in vd]
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    progress(f"input graphs built in {build_s:.1f} s")
    tsegs = [(v, g, e) for v, (g, e) in zip(vd, graphs)]
    sizes = [len(s_) for s_ in segs]

    def plan_now():
        # MOS runs inside the timed step (a host planner over sizes and centroids)
        return rn.mos_plan(sizes, cen) if W.multi else None

    prec0 = {"fp32": rn.FP32, "bf16": rn.BF16, "fp8": rn.FP8}[args.precision]
    p = rn.params(W.R, W.L, W.alpha, metric=W.metric, prec=prec0)
    out = torch.empty((N, W.R), dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()

    for _ in range(args.warmup):
        rn.merge(tsegs, p, plan=plan_now(), out=out)
    torch.cuda.synchronize()

    gpu_id = torch.cuda.get_device_properties(local).uuid
    gpu_id = f"GPU-{gpu_id}" if not str(gpu_id).startswith("GPU-") else str(gpu_id)
    sampler = ClockSampler(gpu_id)
    time.sleep(0.5)
    barrier(dist)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stats = []
    plan_used = None
    ev0.record(stream)
    for _ in range(args.steps):
        torch.cuda.nvtx.range_push("rnsm_merge")
        plan_used = plan_now()
        _, st = rn.merge(tsegs, p, plan=plan_used, out=out)
        torch.cuda.nvtx.range_pop()
        stats.append(st)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(dist)
    clocks = sampler.stop()
    ms = ev0.elapsed_time(ev1)
    ms_max = allmax(dist, ms)
    value = whole_job_rate(N, args.steps, ws, ms_max)

    progress(f"timed steps: {ms / args.steps:.1f} ms per step")
    # roofline of the search kernel (S1, S4, S5 launches), from the
    # library's CUDA events on the launching stream and its NDC counters
    s_bytes = s_ms = 0.0
    launches = 0
    n_search_launches = 0
    for st in stats:
        for i, ph in ((0, 1), (1, 4), (2, 5)):
            s_bytes += (st["search_ndc"][i] * W.dim * 4 + st["search_exp"][i] * W.R * 4 +
                        st["search_queries"][i] * W.dim * 4)
            s_ms += st["phase_ms"][ph]
        launches += st["launches"]
        # one multi-job launch each for S1, S4 and S5 (every pair of the plan)
        n_search_launches += 3
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except OSError:
        pass
    peak = float(peaks.get("hbm_gbs", 6800.0))
    achieved = (s_bytes / n_search_launches) / (s_ms / n_search_launches / 1000.0) / 1e9
    # the committed captures are of the full-size default workload
    full_default = W.name == "sift2x500k" and args.scale == 1.0 and not args.n_per_seg
    traffic = search_profile_traffic() if full_default else None
    search_roof = {"bound": "hbm", "kernel": "search_kernel (S1+S4+S5 launches)",
                   "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                   "peak_source": "measured" if "hbm_gbs" in peaks else "fallback",
                   "traffic": traffic,
                   "algorithmic_bytes_per_launch": s_bytes / n_search_launches,
                   "avg_launch_ms": s_ms / n_search_launches,
                   "l2": search_profile_l2(),
                   "note": "algorithmic bytes; most are served from L2 (see traffic and l2)"}
    # roofline of the S6 source prune, in the unit of its per-owner gather: the
    # owner row and its c = R + c_cross raw pool rows, d x 4 bytes each, per
    # owner (every source vertex), against the measured HBM copy bandwidth
    pool = W.R + (W.L + 1) // 2
    b_per_owner = (pool + 1) * W.dim * 4
    owners = sum(st["pivots"] + st["followers"] for st in stats)
    p_ms = sum(st["phase_ms"][6] for st in stats)
    n_p6 = len(stats) * (len(plan_used) if plan_used else 1)
    p_ach = owners * b_per_owner / (p_ms / 1000.0) / 1e9
    s6_var = stats[-1]["prune_kernel"][0]
    s6_name = (PRUNE_KERNELS[s6_var][0] if pool <= 64 and s6_var in PRUNE_KERNELS
               else "prune_kernel")
    prune_roof = {"bound": "hbm",
                  "kernel": s6_name + " (S6 launches)",
                  "achieved": p_ach, "peak": peak, "unit": "GB/s", "frac": p_ach / peak,
                  "peak_source": "measured" if "hbm_gbs" in peaks else "fallback",
                  "traffic": prune_profile_traffic(s6_var) if full_default else None,
                  "algorithmic_bytes_per_launch": owners * b_per_owner / n_p6,
                  "algorithmic_bytes_per_owner": b_per_owner,
                  "avg_launch_ms": p_ms / n_p6}
    # the same launches as FP32 arithmetic: at most R x c occlusion tests per
    # owner (the walk tests a candidate only against kept ones), 2 FLOP per
    # dimension, against SMs x 128 FP32 lanes x 2 FLOP x the maximum SM clock
    sm_count = torch.cuda.get_device_properties(0).multi_processor_count
    alu_peak = sm_count * 128 * 2 * float(peaks.get("sm_max_mhz", 2070.0)) * 1e6 / 1e12
    f_ach = owners * W.R * pool * W.dim * 2 / (p_ms / 1000.0) / 1e12
    prune_flop = {"bound": "alu", "kernel": prune_roof["kernel"], "achieved_at_most": f_ach,
                  "peak": alu_peak, "unit": "TFLOP/s", "frac_at_most": f_ach / alu_peak,
                  "peak_source": "derived: %d SMs x 128 FP32 lanes x 2 FLOP x %.0f MHz" % (
                      sm_count, float(peaks.get("sm_max_mhz", 2070.0))),
                  "flop_per_owner_at_most": W.R * pool * W.dim * 2,
                  # measured: the FMA pipe's activity in the committed ncu capture
                  "fma_pipe_active_pct_ncu": prune_profile_fma(s6_var) if W.name == "sift2x500k" else None}
    # the dominant kernel family of the FP32 step by live time goes first
    s7_ms = sum(st["phase_ms"][7] for st in stats)
    if p_ms + s7_ms >= s_ms:
        roofline, roofline_other = prune_roof, search_roof
    else:
        roofline, roofline_other = search_roof, prune_roof
    phases = ["validate_init", "S1_expand", "S2_invert", "S3_pivots", "S4_pivot_search",
              "S5_follower_search", "S6_source_prune", "S7_reverse_edges"]
    phase_ms = {nm: sum(st["phase_ms"][i] for st in stats) / len(stats)
                for i, nm in enumerate(phases)}

    # precision pattern: the same merge with BF16 / FP8 prune tiles (tensor
    # cores + FP32 re-decisions); their graphs must equal the FP32 graph
    modes = {}
    ref_out = out.clone()
    for name in W.modes:
        prec = {"bf16": rn.BF16, "fp8": rn.FP8}[name]
        pq = rn.params(W.R, W.L, W.alpha, metric=W.metric, prec=prec)
        oq = torch.empty_like(out)
        for _ in range(1 if huge else 2):
            rn.merge(tsegs, pq, plan=plan_now(), out=oq)
        torch.cuda.synchronize()
        q0, q1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        qs = []
        nq = 1 if huge else max(3, args.steps // 2)
        q0.record(stream)
        for _ in range(nq):
            _, st = rn.merge(tsegs, pq, plan=plan_now(), out=oq)
            qs.append(st)
        q1.record(stream)
        torch.cuda.synchronize()
        qms = q0.elapsed_time(q1) / nq
        modes[name] = {"ms_per_step": qms, "value": N / (qms / 1000.0), "unit": UNIT,
                       "identical_to_fp32": bool(torch.equal(oq, ref_out)),
                       "rechecks_per_step": qs[-1]["rechecks"],
                       "tile_tests_per_step": qs[-1]["tile_tests"],
                       "rechecked_share": (qs[-1]["rechecks"] / qs[-1]["tile_tests"]
                                           if qs[-1]["tile_tests"] else None),
                       # sampled owner distances: tile and FP32 vs FP64, bound use
                       "distance_error": {
                           "tile_vs_fp64_max_rel": qs[-1]["tile_error"][0],
                           "fp32_vs_fp64_max_rel": qs[-1]["tile_error"][1],
                           "tile_vs_fp32_max_share_of_bound": qs[-1]["tile_error"][2],
                           "samples": int(qs[-1]["tile_error"][3])},
                       "prune_ms": round(sum(st["phase_ms"][6] + st["phase_ms"][7]
                                             for st in qs) / nq, 3)}
    if W.multi and not huge:   # (a plan of many groups runs eagerly anyway)
        # batching pattern: S4..S7 of the plan captured once in a CUDA graph, replayed
        pg = rn.params(W.R, W.L, W.alpha, metric=W.metric, flags=rn.FLAG_GRAPH)
        og = torch.empty_like(out)
        for _ in range(2):
            rn.merge(tsegs, pg, plan=plan_now(), out=og)
        torch.cuda.synchronize()
        q0, q1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        nq = max(3, args.steps // 2)
        q0.record(stream)
        for _ in range(nq):
            rn.merge(tsegs, pg, plan=plan_now(), out=og)
        q1.record(stream)
        torch.cuda.synchronize()
        qms = q0.elapsed_time(q1) / nq
        modes["fp32_cuda_graph"] = {"ms_per_step": qms, "value": N / (qms / 1000.0), "unit": UNIT,
                                    "identical_to_fp32": bool(torch.equal(og, ref_out))}
    modes["fp32" if args.precision == "fp32" else args.precision + "_timed_steps"] = {
                     "ms_per_step": ms_max / args.steps,
                     "prune_ms": round(phase_ms["S6_source_prune"] + phase_ms["S7_reverse_edges"], 3)}

    progress("precision modes done")
    # end to end through the public API with host buffers
    in_bytes = sum(v.numel() * 4 for v in vd) + sum(g.numel() * 4 for g, _ in graphs)
    out_bytes = N * W.R * 4
    room = e2e_room(torch, in_bytes, out_bytes)
    if room is not None:
        e2e = {"value": None, "unit": UNIT, "skipped": room}
    else:
        pin_v = [torch.empty(v.shape, dtype=v.dtype, pin_memory=True).copy_(v) for v in vd]
        pin_g = [torch.empty(g.shape, dtype=g.dtype, pin_memory=True).copy_(g) for g, _ in graphs]
        pin_out = torch.empty((N, W.R), dtype=torch.int32).pin_memory()
        dv = [torch.empty_like(v) for v in vd]
        dg = [torch.empty_like(g) for g, _ in graphs]
        h2d = sum(t.numel() * t.element_size() for t in pin_v + pin_g)
        d2h = pin_out.numel() * pin_out.element_size()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier(dist)
        torch.cuda.synchronize()
        e2e_steps = 1 if huge else args.steps
        e0.record(stream)
        for _ in range(e2e_steps):
            for a, b in zip(dv, pin_v):
                a.copy_(b, non_blocking=True)
            for a, b in zip(dg, pin_g):
                a.copy_(b, non_blocking=True)
            rn.merge([(v, g, e) for v, g, (_, e) in zip(dv, dg, graphs)], p, plan=plan_now(),
                     out=out)
            pin_out.copy_(out, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        e2e_ms = allmax(dist, e0.elapsed_time(e1))
        e2e = {"value": whole_job_rate(N, e2e_steps, ws, e2e_ms), "unit": UNIT,
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}
        del pin_v, pin_g, pin_out, dv, dg

    progress(f"e2e: {e2e.get('value')}")
    rec = Xd = None
    if rank == 0 and args.recall_queries > 0:
        Xd = concat_rows(torch, vd)
        big = int(np.argmax(sizes))
        entry = graphs[big][1] + sum(sizes[:big])
        rec = {"ef": 64, "queries": args.recall_queries,
               "value": recall_at_10(rn, torch, W, Xd, out, entry, Q)}
        if W.multi:   # one entry per segment: cross-segment navigation taken out
            offs = np.concatenate([[0], np.cumsum(sizes)])
            rec["value_segment_entries"] = recall_at_10(
                rn, torch, W, Xd, out, [int(graphs[k][1] + offs[k]) for k in range(len(sizes))], Q)

    base = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        base = cpu_baseline(W, args, rn=rn, torch=torch)

    line = None
    if rank == 0:
        vec_bytes = sum(v.numel() * 4 for v in vd)
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic",
                "config": {"workload": W.desc, "segments": sizes,
                           "dim": W.dim, "R": W.R, "L": W.L, "alpha": W.alpha,
                           "metric": "l2" if W.metric == L2_METRIC else "ip",
                           "precision": args.precision,
                           "plan": None if plan_used is None else [list(e[:2]) for e in plan_used],
                           "parallelism": "replicas" if ws > 1 else "single",
                           "l2": f"inputs larger than L2 ({vec_bytes >> 20} MB of vectors)",
                           "input_graph_build_s": round(build_s, 3),
                           "phase_ms": {k: round(v, 3) for k, v in phase_ms.items()},
                           "recall_at_10": rec,
                           "pivots": stats[-1]["pivots"], "followers": stats[-1]["followers"],
                           "ndc_per_step": stats[-1]["ndc"]},
                "clocks": clocks, "e2e": e2e, "gpu_launches": int(launches),
                "precision_modes": modes,
                "roofline": roofline, "roofline_secondary": roofline_other,
                "roofline_prune_flop": prune_flop, "cpu_baseline": base}
    full_headline = W.name == "sift2x500k" and args.scale == 1.0 and not args.n_per_seg
    extra = (rank == 0 and ws == 1 and not args.no_extra and W.name == "sift2x500k" and
             (full_headline or args.extra_scale is not None))
    if extra:
        # the larger workloads, measured after the headline (its memory freed)
        del vd, graphs, tsegs, out, ref_out, Xd
        rn.release_workspace()
        torch.cuda.empty_cache()
        line["extra_workloads"] = run_extra(rn, torch, args.extra_scale or 1.0)
    if rank == 0:
        print(json.dumps(line), flush=True)
    barrier(dist)
    if dist is not None:
        dist.destroy_process_group()
    return 0


EXTRA = (("deep10x2m", 2, 1), ("embed4x250k", 2, 1), ("deep50x100m", 1, 1))
CURVE_EFS = [16, 32, 64, 128, 256]


def run_extra(rn, torch, scale=1.0, nq=1000):
    """The multi-segment workloads at full size, a few steps each: FP32 and
    low-precision ms/step, re-decided tests, graph identity, recall@10; for the
    10-segment DEEP-like workload also the CM comparator and a rebuild by the
    same builder (merge time and recall@10 curves)."""
    res = {}
    for name, steps, warm in EXTRA:
        W = WORKLOADS[name]
        try:
            res[name] = measure_extra(W, rn, torch, steps, warm, nq, scale,
                                      curves=name == "deep10x2m")
        except Exception as e:   # noqa: BLE001 -- one workload's failure is reported, not fatal
            res[name] = {"error": f"{type(e).__name__}: {e}"}
        rn.release_workspace()
        torch.cuda.empty_cache()
        progress(f"extra workload {name} done")
    return res


def measure_extra(W, rn, torch, steps, warm, nq, scale=1.0, curves=False):
    segs, Q = W.make(scale, nq)
    vd = [s_ if torch.is_tensor(s_) else torch.from_numpy(s_).cuda() for s_ in segs]
    del segs
    sizes = [int(v.shape[0]) for v in vd]
    N = sum(sizes)
    cen = centroids_of(vd)
    progress(f"{W.name}: {len(vd)} segments, {N} rows on the device")
    t0 = time.perf_counter()
    graphs = [rn.build_segment(v, W.R, W.L, W.alpha, metric=W.metric) for v in vd]
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    tsegs = [(v, g, e) for v, (g, e) in zip(vd, graphs)]
    stream = torch.cuda.current_stream()

    def timed(p, out):
        for _ in range(warm):
            rn.merge(tsegs, p, plan=rn.mos_plan(sizes, cen), out=out)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            _, st = rn.merge(tsegs, p, plan=rn.mos_plan(sizes, cen), out=out)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps, st

    out = torch.empty((N, W.R), dtype=torch.int32, device="cuda")
    ms32, st32 = timed(rn.params(W.R, W.L, W.alpha, metric=W.metric), out)
    r = {"workload": W.desc, "scale": scale, "segments": sizes,
         "plan_edges": len(rn.mos_plan(sizes, cen)),
         "steps": steps, "warmup": warm, "input_graph_build_s": round(build_s, 3),
         "fp32": {"ms_per_step": ms32, "value": N / (ms32 / 1000.0), "unit": UNIT,
                  "phase_ms": [round(x, 3) for x in st32["phase_ms"]],
                  "prune_kernel_s6_s7": list(st32["prune_kernel"])}}
    if curves:
        # the batching pattern's effect: the same merge with one search launch per
        # plan edge (RNSM_SEARCH_PER_JOB=1) instead of one launch per phase over
        # every edge of the plan; same queries, same graph
        oj = torch.empty_like(out)
        os.environ["RNSM_SEARCH_PER_JOB"] = "1"
        try:
            msj, stj = timed(rn.params(W.R, W.L, W.alpha, metric=W.metric), oj)
        finally:
            del os.environ["RNSM_SEARCH_PER_JOB"]
        srch = lambda st: round(st["phase_ms"][1] + st["phase_ms"][4] + st["phase_ms"][5], 3)
        r["batching"] = {"one_launch_per_phase_ms_per_step": ms32,
                         "one_launch_per_edge_ms_per_step": msj,
                         "search_ms_one_launch_per_phase": srch(st32),
                         "search_ms_one_launch_per_edge": srch(stj),
                         "launches_one_per_phase": int(st32["launches"]),
                         "launches_one_per_edge": int(stj["launches"]),
                         "identical": bool(torch.equal(oj, out))}
        del oj
    oq = torch.empty_like(out)
    for name in W.modes:
        prec = {"bf16": rn.BF16, "fp8": rn.FP8}[name]
        msq, stq = timed(rn.params(W.R, W.L, W.alpha, metric=W.metric, prec=prec), oq)
        r[name] = {"ms_per_step": msq, "value": N / (msq / 1000.0), "unit": UNIT,
                   "identical_to_fp32": bool(torch.equal(oq, out)),
                   "rechecks_per_step": int(stq["rechecks"]),
                   "tile_tests_per_step": int(stq["tile_tests"]),
                   "rechecked_share": (stq["rechecks"] / stq["tile_tests"] if stq["tile_tests"] else None),
                   "tile_vs_fp32_max_share_of_bound": stq["tile_error"][2],
                   "prune_ms": round(stq["phase_ms"][6] + stq["phase_ms"][7], 3)}
    del oq
    Xd = concat_rows(torch, vd)
    Qd = (Q if torch.is_tensor(Q) else torch.from_numpy(Q)).cuda()
    big = int(np.argmax(sizes))
    offs = np.concatenate([[0], np.cumsum(sizes)])
    entry = int(graphs[big][1] + offs[big])
    efs = CURVE_EFS if curves else [64]
    gt = None

    def curve(adj, ent):
        nonlocal gt
        if gt is None:
            def native(rows64, q64):
                if W.metric == L2_METRIC:
                    return ((rows64 - q64[:, None, :]) ** 2).sum(-1)
                return 1.0 - (rows64 * q64[:, None, :]).sum(-1)
            gt = true_d10(torch, W, Xd, Qd, native)
        return dict(zip(map(str, efs), recall_at_10(rn, torch, W, Xd, adj, ent, Qd, ef=efs, gt=gt)))

    r["recall_at_10"] = {"queries": nq, "rnsm": curve(out, entry)}
    if curves:
        # the CM comparator (every source vertex a naive search) on the same plan
        oc = torch.empty_like(out)
        msc, stc = timed(rn.params(W.R, W.L, W.alpha, metric=W.metric, flags=rn.FLAG_CM), oc)
        r["cm"] = {"ms_per_step": msc, "value": N / (msc / 1000.0), "unit": UNIT,
                   "naive_searches": int(stc["pivots"]), "rnsm_over_cm_speedup": msc / ms32}
        r["recall_at_10"]["cm"] = curve(oc, entry)
        del oc
        # a rebuild of all rows by the same builder
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        gr, er = rn.build_segment(Xd, W.R, W.L, W.alpha, metric=W.metric)
        torch.cuda.synchronize()
        rb_s = time.perf_counter() - t0
        r["rebuild"] = {"s": rb_s, "rnsm_over_rebuild_speedup": rb_s / (ms32 / 1000.0)}
        r["recall_at_10"]["rebuild"] = curve(gr, int(er))
        r["recall_at_10"]["rnsm_segment_entries"] = curve(
            out, [int(graphs[k][1] + offs[k]) for k in range(len(sizes))])
        del gr
        # denser merge plans on the same inputs: Algorithm 3 with a larger degree
        # bound, and every pair once (the edges of the complete merge graph in the
        # plan's execution order: closer pairs first, smaller into larger)
        m = len(sizes)
        cost = {(a, b): float(np.linalg.norm(cen[a].astype(np.float64) - cen[b]))
                for a in range(m) for b in range(a + 1, m)}
        allp = sorted(cost, key=lambda e: (cost[e], e))
        allp = [((b, a) if sizes[b] < sizes[a] or (sizes[a] == sizes[b]) else (a, b)) + (cost[(a, b)],)
                for a, b in allp]
        for name, plan in (("rnsm_mos_degree6", rn.mos_plan(sizes, cen, degree_bound=6)),
                           ("rnsm_all_pairs", allp)):
            op = torch.empty_like(out)
            pp = rn.params(W.R, W.L, W.alpha, metric=W.metric)
            rn.merge(tsegs, pp, plan=plan, out=op)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rn.merge(tsegs, pp, plan=plan, out=op)
            e1.record(stream)
            torch.cuda.synchronize()
            r[name] = {"plan_edges": len(plan), "ms_per_step": e0.elapsed_time(e1)}
            r["recall_at_10"][name] = curve(op, entry)
            del op
    del out, tsegs, graphs, vd, Xd
    return r


def run_incremental(args, ws, rank, local):
    """Incremental merging: partition 0's graph is the index; partitions 1..9 are
    merged into it one at a time (each merge: the new partition is the source,
    the index the target).  One step = the whole sequence of nine merges; value =
    vertices of the merged graphs per second (sum over the nine merges)."""
    import torch

    from paper_2602_17099_gb300 import build as pkg_build
    from paper_2602_17099_gb300 import rnsm as rn

    W = WORKLOADS[args.workload]
    dist = init_dist(ws)
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device (there is no CPU path)")
    torch.cuda.set_device(local)
    if rank == 0 or ws == 1:
        pkg_build.build()
    barrier(dist)
    rn.lib()
    segs, Q, allx = W.make(args.scale, args.recall_queries)
    m, n_part = len(segs), len(segs[0])
    progress(f"{W.name}: {m} partitions of {n_part} rows on the device")
    t0 = time.perf_counter()
    graphs = [rn.build_segment(v, W.R, W.L, W.alpha, metric=W.metric) for v in segs]
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    progress(f"partition graphs built in {build_s:.1f} s")
    bufs = [torch.empty((m * n_part, W.R), dtype=torch.int32, device="cuda") for _ in range(2)]

    def sequence(p):
        g, e = graphs[0]
        n_idx, stats = n_part, []
        for k in range(1, m):
            out = bufs[k % 2][:n_idx + n_part]
            g, st = rn.merge([(allx[:n_idx], g, e), (segs[k], graphs[k][0], graphs[k][1])], p,
                             plan=[(1, 0, 0.0)], out=out)
            stats.append(st)
            n_idx += n_part
        return g, e, stats

    units = sum((k + 1) * n_part for k in range(1, m))   # vertices of the nine merged graphs
    p = rn.params(W.R, W.L, W.alpha, metric=W.metric)
    for _ in range(args.warmup):
        sequence(p)
    torch.cuda.synchronize()
    gpu_id = torch.cuda.get_device_properties(local).uuid
    gpu_id = f"GPU-{gpu_id}" if not str(gpu_id).startswith("GPU-") else str(gpu_id)
    sampler = ClockSampler(gpu_id)
    time.sleep(0.5)
    barrier(dist)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        final, entry, stats = sequence(p)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(dist)
    clocks = sampler.stop()
    ms = allmax(dist, ev0.elapsed_time(ev1))
    value = whole_job_rate(units, args.steps, ws, ms)
    progress(f"timed sequences: {ms / args.steps:.1f} ms each")
    per_merge = [round(sum(st["phase_ms"]), 3) for st in stats]
    launches = sum(st["launches"] for st in stats) * args.steps
    ref = final.clone()
    modes = {}
    for name in W.modes:
        prec = {"bf16": rn.BF16, "fp8": rn.FP8}[name]
        pq = rn.params(W.R, W.L, W.alpha, metric=W.metric, prec=prec)
        sequence(pq)
        torch.cuda.synchronize()
        q0, q1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        q0.record(stream)
        fq, _, sq = sequence(pq)
        q1.record(stream)
        torch.cuda.synchronize()
        qms = q0.elapsed_time(q1)
        modes[name] = {"ms_per_step": qms, "value": units / (qms / 1000.0), "unit": UNIT,
                       "identical_to_fp32": bool(torch.equal(fq, ref)),
                       "rechecks_per_step": int(sum(st["rechecks"] for st in sq))}
    # the multi-pair union variant: the partitions merged three at a time (each
    # into the index, the later ones also into the earlier ones), one prune per
    # source vertex and one reverse-edge pass per step
    def sequence_union(p, group=3):
        g, e = graphs[0]
        n_idx, nstep = n_part, 0
        for k0 in range(1, m, group):
            ks = list(range(k0, min(m, k0 + group)))
            plan = [(i + 1, 0, 0.0) for i in range(len(ks))]
            plan += [(j + 1, i + 1, 0.0) for i in range(len(ks)) for j in range(i + 1, len(ks))]
            out = bufs[nstep % 2][:n_idx + len(ks) * n_part]
            g, _ = rn.merge([(allx[:n_idx], g, e)] + [(segs[k], graphs[k][0], graphs[k][1]) for k in ks],
                            p, plan=plan, out=out)
            n_idx += len(ks) * n_part
            nstep += 1
        return g
    pu = rn.params(W.R, W.L, W.alpha, metric=W.metric, flags=rn.FLAG_UNION)
    sequence_union(pu)
    torch.cuda.synchronize()
    q0, q1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    q0.record(stream)
    fu = sequence_union(pu)
    q1.record(stream)
    torch.cuda.synchronize()
    union = {"ms_per_sequence": q0.elapsed_time(q1), "merges": (m - 1 + 2) // 3,
             "note": "three partitions per merge call (RNSM_FLAG_UNION); sequential: nine calls"}
    rec = None
    if args.recall_queries > 0:
        rec = recall_at_10(rn, torch, W, allx, ref, entry, Q[:args.recall_queries])
        union["recall_at_10"] = recall_at_10(rn, torch, W, allx, fu, entry, Q[:args.recall_queries])
    modes["union3"] = union
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic (seeded; no dataset)",
                "config": {"workload": W.desc, "partitions": m, "rows_per_partition": n_part,
                           "dim": W.dim, "R": W.R, "L": W.L, "alpha": W.alpha, "metric": "l2",
                           "precision": "fp32", "parallelism": "replicas" if ws > 1 else "single",
                           "l2": "inputs larger than L2 (%d MB of vectors)" % (allx.numel() * 4 >> 20),
                           "partition_graph_build_s": round(build_s, 3),
                           "merge_ms_by_index_size": per_merge, "recall_at_10": rec},
                "clocks": clocks, "gpu_launches": int(launches),
                "e2e": {"value": None, "unit": UNIT,
                        "skipped": "device-resident stream; the default workload carries e2e"},
                "precision_modes": modes, "roofline": None, "cpu_baseline": None}
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
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="sift2x500k")
    ap.add_argument("--scale", type=float, default=1.0,
                    help="size factor of the workload (1.0 = full size)")
    ap.add_argument("--n-per-seg", type=int, default=0,
                    help="sift2x500k only: rows per segment (overrides --scale)")
    ap.add_argument("--recall-queries", type=int, default=1000)
    ap.add_argument("--precision", choices=["fp32", "bf16", "fp8"], default="fp32",
                    help="prune tiles of the timed steps (the headline is FP32; the other "
                         "modes are measured beside it either way)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the multi-segment workloads the default run also measures")
    ap.add_argument("--extra-scale", type=float, default=None,
                    help="size factor of those workloads (default: full size, measured only "
                         "after the full-size default workload)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    ws, rank, local = dist_env()
    if args.impl == "reference":
        if args.workload == "incr10x1m":
            if rank == 0:
                print(json.dumps({"impl": "reference", "unavailable": "the incremental workload has "
                                  "no oracle arm (its sequence is checked against the oracle in "
                                  "tests/test_gpu_parity.py)"}), flush=True)
            return 0
        return run_reference(args, ws, rank)
    if args.workload == "incr10x1m":
        return run_incremental(args, ws, rank, local)
    return run_ours(args, ws, rank, local)


if __name__ == "__main__":
    sys.exit(main())
