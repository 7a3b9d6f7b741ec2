"""The benchmark's multi-rank path (independent replicas, one per GPU):
barrier, max-over-ranks timing and whole-job aggregation, exercised with two
gloo ranks on the CPU."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import bench
    ws, r, _ = bench.dist_env()
    dist = bench.init_dist(ws)
    bench.barrier(dist)
    slowest = bench.allmax(dist, 10.0 * (r + 1))      # rank 1 is the slow one
    rate = bench.whole_job_rate(1000, 4, ws, slowest)
    bench.barrier(dist)
    dist.destroy_process_group()
    q.put((r, slowest, rate))


def test_two_gloo_ranks_take_the_slowest_rank_and_sum_units():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=5) for _ in range(2))
    for r, slowest, rate in got:
        assert slowest == 20.0                      # max over ranks
        assert rate == pytest.approx(1000 * 4 * 2 / 0.020)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.init_dist(1) is None
    assert bench.allmax(None, 3.5) == 3.5
    assert bench.whole_job_rate(10, 2, 1, 1000.0) == 20.0


def test_profile_traffic_only_for_matching_sources(tmp_path):
    # the committed ncu summaries give per-launch DRAM bytes only while the
    # kernel sources they were taken on are unchanged (sha256 prefix)
    import hashlib
    sys.path.insert(0, ROOT)
    import bench
    src = tmp_path / "k.cu"
    src.write_bytes(b"__global__ void k() {}\n")
    h = hashlib.sha256(src.read_bytes()).hexdigest()[:16]
    prof = tmp_path / "p.txt"
    prof.write_text(f"# title\n\nsources sha256[:16]: {h}\nbytes per launch: 123456\n")
    assert bench.profile_traffic(str(prof), [str(src)], "sources sha256[:16]",
                                 "bytes per launch") == 123456.0
    src.write_bytes(b"__global__ void k() { }\n")          # the kernel changed
    assert bench.profile_traffic(str(prof), [str(src)], "sources sha256[:16]",
                                 "bytes per launch") is None
    assert bench.profile_traffic(str(tmp_path / "none.txt"), [str(src)], "a", "b") is None


def test_committed_profiles_match_the_current_sources():
    # the bench reads DRAM traffic, L2 and FMA-pipe figures from the committed ncu
    # summaries only while they were taken on the current kernel sources
    sys.path.insert(0, ROOT)
    import bench
    assert bench.prune_profile_traffic() is not None
    assert bench.search_profile_traffic() is not None
    assert bench.prune_profile_fma() is not None
    l2 = bench.search_profile_l2()
    assert l2 and 0 < l2["l2_hit_rate_pct"] <= 100 and 0 < l2["l2_throughput_pct"] <= 100
