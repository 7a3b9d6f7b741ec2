"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Integer-valued (SIFT-like) inputs make every FP32 distance exact, so there
the GPU must equal the oracle bit for bit.  On real-valued inputs distances
must agree within a relative 1e-5, and result lists must agree except where
the oracle logged a decision closer than that bound (a near tie)."""
import numpy as np
import pytest
import torch

import oracle
from workloads import generators as gen

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(scope="module")
def rn():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_17099_gb300 import build as b
    b.build()
    from paper_2602_17099_gb300 import rnsm
    return rnsm


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    return t.cpu().numpy()


_cache = {}


def sift_graph(n, d=128, R=32, L=64, seed=3):
    key = ("sift", n, d, R, L, seed)
    if key not in _cache:
        X = gen.sift_like(n, seed, d=d)
        adj, ep = oracle.build_graph(X, R, L, 1.2)
        _cache[key] = (X, adj, ep)
    return _cache[key]


def gauss_graph(n, d=32, R=16, L=32, seed=1):
    key = ("gauss", n, d, R, L, seed)
    if key not in _cache:
        X = gen.gaussian(n, d, seed)
        adj, ep = oracle.build_graph(X, R, L, 1.2)
        _cache[key] = (X, adj, ep)
    return _cache[key]


# ------------------------------------------------------------------ search

@pytest.mark.parametrize("ef,k,nseed", [(1, 1, 1), (17, 16, 1), (32, 10, 1), (64, 64, 1),
                                        (100, 50, 3), (200, 200, 40), (256, 7, 64)])
def test_search_exact_on_integer_data(rn, ef, k, nseed):
    X, adj, ep = sift_graph(6000)
    Q = gen.sift_like(517, 99, d=128)           # ragged: not a multiple of the warp count
    rng = np.random.default_rng(ef)
    seeds = rng.integers(-1, len(X), size=(len(Q), nseed)).astype(np.int32)
    seeds[:, 0] = ep
    want, wd, wndc, _, _ = oracle.beam_search(X, adj, Q, seeds, ef, k)
    ids, dd, ndc = rn.search(dev(X), dev(adj), dev(Q), dev(seeds), ef, k, want_ndc=True)
    np.testing.assert_array_equal(host(ids), want)
    ok = want >= 0
    np.testing.assert_array_equal(host(dd)[ok], wd[ok].astype(np.float32))
    # the visited hash is exact until it overflows: NDC can only exceed the
    # oracle's, and overflows must stay rare
    assert (host(ndc) >= wndc).all()
    assert host(ndc).sum() <= 1.01 * wndc.sum()


@pytest.mark.parametrize("metric", [oracle.L2, oracle.IP])
def test_search_float_data_within_tolerance(rn, metric):
    if metric == oracle.L2:
        X, adj, ep = gauss_graph(5000)
        Q = gen.gaussian(1000, 32, 2)
    else:
        X = gen.deep_like(5000, 21, d=96)
        adj, ep = oracle.build_graph(X, 16, 32, 1.2, metric=oracle.IP)
        Q = gen.deep_like(1000, 22, d=96)
    seeds = np.full((len(Q), 1), ep, np.int32)
    want, wd, _, _, margin = oracle.beam_search(X, adj, Q, seeds, 48, 32, metric)
    ids, dd, _ = rn.search(dev(X), dev(adj), dev(Q), dev(seeds), 48, 32, metric=metric)
    ids, dd = host(ids), host(dd)
    same = (ids == want).all(axis=1)
    decided = margin > TOL
    assert same[decided].all(), f"{(~same[decided]).sum()} decided queries differ"
    # distances of identical ids agree within the relative bound
    m = (ids == want) & (want >= 0)
    rel = np.abs(dd[m] - wd[m]) / np.maximum(np.abs(wd[m]), 1e-30)
    if metric == oracle.IP:   # 1 - <x,y>: the error is absolute in <x,y>
        rel = np.abs(dd[m] - wd[m])
    assert rel.max() <= TOL
    assert same.mean() > 0.97


def test_search_edge_cases(rn):
    # one vertex; an empty graph (no edges); seeds all -1; duplicates of the entry
    X = gen.sift_like(50, 7, d=32)
    empty = np.full((50, 8), -1, np.int32)
    Q = X[:5].copy()
    seeds = np.array([[3, 3, -1], [-1, -1, -1], [0, 1, 2], [49, 48, 47], [10, -1, 10]], np.int32)
    want, _, _, _, _ = oracle.beam_search(X, empty, Q, seeds, 4, 4)
    ids, _, _ = rn.search(dev(X), dev(empty), dev(Q), dev(seeds), 4, 4)
    np.testing.assert_array_equal(host(ids), want)
    one = X[:1].copy()
    ids, _, _ = rn.search(dev(one), dev(np.full((1, 4), -1, np.int32)), dev(Q), dev(
        np.zeros((5, 1), np.int32)), 8, 3)
    assert (host(ids)[:, 0] == 0).all() and (host(ids)[:, 1:] == -1).all()


def test_expand_exact_on_integer_data(rn):
    X, adj, _ = sift_graph(6000)
    want, _, _, _ = oracle.expand(X, adj, 16)
    got = rn.expand(dev(X), dev(adj), 16)
    np.testing.assert_array_equal(host(got), want)


def test_reverse_knn_bit_exact(rn):
    X, adj, _ = sift_graph(6000)
    nplus, _, _, _ = oracle.expand(X, adj, 16)
    for k in (1, 5, 16):
        wo, wi = oracle.reverse_knn(nplus, k)
        go, gi = rn.reverse_knn(dev(nplus), k)
        np.testing.assert_array_equal(host(go), wo)
        np.testing.assert_array_equal(host(gi), wi)


# ------------------------------------------------------------------- prune

def _pools(n, w, seed, nown):
    rng = np.random.default_rng(seed)
    owners = rng.choice(n, nown, replace=False).astype(np.int32)
    pool = rng.integers(-1, n, size=(nown, w)).astype(np.int32)
    pool[:, 3] = owners          # the owner itself must be dropped
    pool[:, 5] = pool[:, 4]      # duplicates must be dropped
    return owners, pool


@pytest.mark.parametrize("R,w,alpha", [(32, 64, 1.2), (16, 40, 1.0), (8, 200, 1.2),
                                       (64, 128, 1.5), (32, 1000, 1.2), (5, 7, 2.0)])
def test_prune_exact_on_integer_data(rn, R, w, alpha):
    X = gen.sift_like(3000, 5, d=128)
    owners, pool = _pools(3000, w, R + w, 301)
    want, _ = oracle.prune(X, owners.astype(np.int64), pool, R, alpha)
    got = rn.prune(dev(X), dev(owners), dev(pool), R, alpha)
    np.testing.assert_array_equal(host(got), want)
    want2, _ = oracle.prune(X, owners.astype(np.int64), pool, R, alpha, keep_all_if_fit=True)
    got2 = rn.prune(dev(X), dev(owners), dev(pool), R, alpha, keep_all_if_fit=True)
    np.testing.assert_array_equal(host(got2), want2)


@pytest.mark.parametrize("d", [32, 96, 768])
def test_prune_float_data_within_tolerance(rn, d):
    X = gen.gaussian(2000, d, 9) if d == 32 else gen.deep_like(2000, 9, d=d)
    owners, pool = _pools(2000, 96, d, 500)
    want, margin = oracle.prune(X, owners.astype(np.int64), pool, 32, 1.2)
    got = host(rn.prune(dev(X), dev(owners), dev(pool), 32, 1.2))
    same = (got == want).all(axis=1)
    assert same[margin > TOL].all()
    assert same.mean() > 0.97


def test_reverse_edges_exact_on_integer_data(rn):
    X, adj, _ = sift_graph(6000)
    n = len(X)
    rng = np.random.default_rng(4)
    ne = 40000
    eu = rng.integers(0, n, ne).astype(np.int32)
    ev = rng.integers(0, n, ne).astype(np.int32)
    hub = eu[:3000].copy()
    hub[:] = 17                   # one target with a large incoming pool
    eu[:3000] = hub
    keep = eu != ev
    eu, ev = eu[keep], ev[keep]
    pairs = np.unique(np.stack([eu, ev], 1), axis=0)
    eu, ev = pairs[:, 0].copy(), pairs[:, 1].copy()
    lists = adj.copy()
    want = oracle.reverse_edges(X, lists, eu, ev, 1.2)
    got = rn.reverse_edges(dev(X), dev(lists), dev(eu), dev(ev), 1.2)
    np.testing.assert_array_equal(host(got), want)


def test_medoid_matches_oracle(rn):
    for X in (gen.sift_like(7777, 8, d=128), gen.gaussian(5000, 32, 3)):
        assert rn.medoid(dev(X)) == oracle.medoid(X)


def test_build_segment_exact_on_integer_data(rn):
    X = gen.sift_like(4000, 12, d=32)
    for bm in (64, 300):
        want, wep = oracle.build_graph(X, 16, 32, 1.2, batch_max=bm)
        got, gep = rn.build_segment(dev(X), 16, 32, 1.2, batch_max=bm)
        assert gep == wep
        np.testing.assert_array_equal(host(got), want)


# ------------------------------------------------------------------- merge

def _merge_both(rn, segs, graphs, entries, plan, R, L, **kw):
    want, wst = oracle.rnsm_merge(segs, graphs, entries, [(a, b) for a, b, *_ in plan], R, L, 1.2,
                                  **kw)
    p = rn.params(R, L, 1.2, **{k: v for k, v in kw.items() if k in
                                ("k_rev", "k_plus", "ef_slide", "c_cross", "metric")})
    tsegs = [(dev(s), dev(g), e) for s, g, e in zip(segs, graphs, entries)]
    got, gst = rn.merge(tsegs, p, plan)
    return host(got), want, gst, wst


def test_merge_pair_exact_on_integer_data(rn):
    segs = [gen.sift_like(5000, 31, d=128), gen.sift_like(3100, 32, d=128)]
    gs = [oracle.build_graph(s, 32, 64, 1.2) for s in segs]
    got, want, gst, wst = _merge_both(rn, segs, [g for g, _ in gs], [e for _, e in gs],
                                      [(1, 0)], 32, 64)
    np.testing.assert_array_equal(got, want)
    assert gst["pivots"] == wst["pivots"] and gst["followers"] == wst["followers"]
    assert gst["reverse_edges"] == wst["reverse_edges"]
    assert gst["ndc"] >= wst["ndc_expand"] + wst["ndc_search"]


def test_merge_default_plan_and_parameters(rn):
    segs = [gen.sift_like(1200, 41, d=32), gen.sift_like(1500, 42, d=32)]
    gs = [oracle.build_graph(s, 16, 32, 1.2) for s in segs]
    for kw in ({}, {"k_rev": 3, "k_plus": 8, "ef_slide": 20, "c_cross": 10}):
        want, _ = oracle.rnsm_merge(segs, [g for g, _ in gs], [e for _, e in gs], [(0, 1)], 16, 32,
                                    1.2, **kw)
        tsegs = [(dev(s), dev(g), e) for s, (g, e) in zip(segs, gs)]
        got, _ = rn.merge(tsegs, rn.params(16, 32, 1.2, **kw))   # plan=None: smaller -> larger
        np.testing.assert_array_equal(host(got), want)


def test_merge_multi_segment_plan_exact(rn):
    sizes = [900, 1400, 600, 1100]
    segs = [gen.sift_like(n, 50 + i, d=32) for i, n in enumerate(sizes)]
    gs = [oracle.build_graph(s, 16, 32, 1.2) for s in segs]
    cen = np.stack([s.astype(np.float64).mean(0) for s in segs]).astype(np.float32)
    plan = oracle.mos_plan(sizes, cen)
    assert plan == rn.mos_plan(sizes, cen)
    got, want, _, _ = _merge_both(rn, segs, [g for g, _ in gs], [e for _, e in gs], plan, 16, 32)
    np.testing.assert_array_equal(got, want)


def test_incremental_merge_matches_oracle_step_by_step(rn):
    # incremental merging (Exp-5's scenario): partition 0's graph is the index;
    # every next partition is merged into it as the source, and the merged graph
    # (global ids = index ids, then the partition's) is the next step's index
    parts = [gen.sift_like(n, 80 + i, d=32) for i, n in enumerate([700, 500, 650, 400])]
    gs = [oracle.build_graph(s, 12, 24, 1.2) for s in parts]
    idx_x, (idx_g, idx_e) = parts[0], gs[0]
    d_idx_g = dev(idx_g)
    for k in range(1, len(parts)):
        want, _ = oracle.rnsm_merge([idx_x, parts[k]], [idx_g, gs[k][0]], [idx_e, gs[k][1]],
                                    [(1, 0)], 12, 24, 1.2)
        got, _ = rn.merge([(dev(idx_x), d_idx_g, idx_e), (dev(parts[k]), dev(gs[k][0]), gs[k][1])],
                          rn.params(12, 24, 1.2), [(1, 0, 0.0)])
        np.testing.assert_array_equal(host(got), want)
        idx_x, idx_g, d_idx_g = np.concatenate([idx_x, parts[k]]), want, got


def test_merge_tiny_segments_exact(rn):
    # segments of 1, 9 and 15 vertices (fewer than the query schedule's smallest
    # locality bucket, one vertex without edges), in FP32 and BF16
    sizes = [1, 9, 15]
    segs = [gen.sift_like(n, 70 + i, d=32) for i, n in enumerate(sizes)]
    gs = [oracle.build_graph(s, 4, 8, 1.2) for s in segs]
    plan = [(1, 0), (0, 2), (1, 2)]
    want, _ = oracle.rnsm_merge(segs, [g for g, _ in gs], [e for _, e in gs], plan, 4, 8, 1.2)
    tsegs = [(dev(sg), dev(g), e) for sg, (g, e) in zip(segs, gs)]
    for prec in (rn.FP32, rn.BF16):
        got, _ = rn.merge(tsegs, rn.params(4, 8, 1.2, prec=prec), [(a, b, 0.0) for a, b in plan])
        np.testing.assert_array_equal(host(got), want)


@pytest.mark.parametrize("flags,per_job", [(0, False), (2, False), (0, True)])
def test_merge_batched_plan_with_shared_sources_exact(rn, monkeypatch, flags, per_job):
    # six uneven segments, a hand-made plan where sources serve several edges and
    # segments are source and target in turn: the batched executor (all S1 in
    # one launch, all S4 and all S5 of the plan in one launch each) must give
    # Algorithm 2 applied edge by edge; so must one search launch per plan edge
    # (RNSM_SEARCH_PER_JOB=1, the batching measurement's comparison)
    if per_job:
        monkeypatch.setenv("RNSM_SEARCH_PER_JOB", "1")
    sizes = [700, 1300, 450, 1000, 820, 1600]
    segs = [gen.sift_like(n, 60 + i, d=64) for i, n in enumerate(sizes)]
    gs = [oracle.build_graph(s, 16, 32, 1.2) for s in segs]
    plan = [(2, 0), (2, 1), (0, 1), (4, 3), (1, 5), (3, 5), (2, 4), (0, 3), (4, 5)]
    want, wst = oracle.rnsm_merge(segs, [g for g, _ in gs], [e for _, e in gs], plan, 16, 32, 1.2)
    tsegs = [(dev(sg), dev(g), e) for sg, (g, e) in zip(segs, gs)]
    got, gst = rn.merge(tsegs, rn.params(16, 32, 1.2, flags=flags), [(a, b, 0.0) for a, b in plan])
    np.testing.assert_array_equal(host(got), want)
    assert gst["reverse_edges"] == wst["reverse_edges"]
    assert gst["pivots"] == wst["pivots"] and gst["followers"] == wst["followers"]


def test_merge_graph_mode_captures_then_replays(rn):
    # RNSM_FLAG_GRAPH: the first call captures S4..S7 of the plan in a CUDA graph,
    # the second replays it; both equal the eager executor
    sizes = [800, 1200, 650, 1000]
    segs = [gen.sift_like(n, 70 + i, d=32) for i, n in enumerate(sizes)]
    gs = [oracle.build_graph(s, 16, 32, 1.2) for s in segs]
    plan = [(2, 0), (0, 1), (3, 1), (2, 3)]
    tsegs = [(dev(sg), dev(g), e) for sg, (g, e) in zip(segs, gs)]
    cplan = [(a, b, 0.0) for a, b in plan]
    want, sw = rn.merge(tsegs, rn.params(16, 32, 1.2), cplan)
    got1, s1 = rn.merge(tsegs, rn.params(16, 32, 1.2, flags=rn.FLAG_GRAPH), cplan)
    got2, s2 = rn.merge(tsegs, rn.params(16, 32, 1.2, flags=rn.FLAG_GRAPH), cplan)
    np.testing.assert_array_equal(host(got1), host(want))
    np.testing.assert_array_equal(host(got2), host(want))
    for st in (s1, s2):
        assert st["reverse_edges"] == sw["reverse_edges"] and st["ndc"] == sw["ndc"]
        assert st["pivots"] == sw["pivots"]
    assert s2["launches"] == s1["launches"] > 0
    ref, _ = oracle.rnsm_merge(segs, [g for g, _ in gs], [e for _, e in gs], plan, 16, 32, 1.2)
    np.testing.assert_array_equal(host(got2), ref)


def test_merge_float_data_recall_within_tolerance(rn):
    segs, Q = gen.tiny_case()
    gs = [oracle.build_graph(s, 16, 32, 1.2) for s in segs]
    got, want, _, _ = _merge_both(rn, segs, [g for g, _ in gs], [e for _, e in gs], [(1, 0)], 16,
                                  32)
    X = np.concatenate(segs)
    _, gd = oracle.bruteforce_knn(X, Q, 10)
    ep = np.full((len(Q), 1), gs[0][1], np.int32)
    for ef in (16, 32, 64):
        rw = oracle.recall_at_k(oracle.beam_search(X, want, Q, ep, ef, 10)[0], X, gd, Q)
        rg = oracle.recall_at_k(oracle.beam_search(X, got, Q, ep, ef, 10)[0], X, gd, Q)
        assert abs(rw - rg) <= 0.005, (ef, rw, rg)
    assert (got == want).all(axis=1).mean() > 0.9


def test_merge_cm_flag_runs_every_vertex_as_pivot(rn):
    segs = [gen.sift_like(800, 61, d=32), gen.sift_like(900, 62, d=32)]
    gs = [oracle.build_graph(s, 16, 32, 1.2) for s in segs]
    tsegs = [(dev(s), dev(g), e) for s, (g, e) in zip(segs, gs)]
    got, st = rn.merge(tsegs, rn.params(16, 32, 1.2, flags=rn.FLAG_CM))
    assert st["pivots"] == 800 and st["followers"] == 0


# ------------------------------------------------------------- validation

def test_device_validation_errors(rn):
    X = gen.sift_like(100, 1, d=32)
    adj, ep = oracle.build_graph(X, 8, 16, 1.2)
    bad = adj.copy()
    bad[5, 2] = 100
    with pytest.raises(rn.RnsmError) as e:
        rn.merge([(dev(X), dev(bad), ep), (dev(X), dev(adj), ep)], rn.params(8, 16))
    assert e.value.status == rn.EGRAPH
    Xn = X.copy()
    Xn[7, 3] = np.nan
    with pytest.raises(rn.RnsmError) as e:
        rn.merge([(dev(Xn), dev(adj), ep), (dev(X), dev(adj), ep)], rn.params(8, 16))
    assert e.value.status == rn.EGRAPH
    with pytest.raises(rn.RnsmError) as e:
        rn.search(dev(X), dev(adj), dev(X[:3]), dev(np.array([[0], [100], [1]], np.int32)), 8, 4)
    assert e.value.status == rn.EGRAPH


# ------------------------------------------------------------- pivots (S3)

@pytest.mark.parametrize("seed,k", [(0, 1), (1, 3), (2, 5), (3, 7), (4, 16)])
def test_device_pivot_selection_equals_lazy_greedy(rn, seed, k):
    X = gen.sift_like(4000, 70 + seed, d=32) if seed % 2 else gen.gaussian(4000, 16, 70 + seed)
    adj, _ = oracle.build_graph(X, 16, 32, 1.2)
    nplus, _, _, _ = oracle.expand(X, adj, 16)
    offs, ids = oracle.reverse_knn(nplus, k)
    want_of, want_piv, _ = oracle.select_pivots(len(X), offs, ids)
    got_of, npiv, rounds = rn.select_pivots_gpu(dev(nplus), k, dev(offs),
                                                dev(ids if len(ids) else np.zeros(1, np.int32)))
    np.testing.assert_array_equal(host(got_of), want_of)
    assert npiv == len(want_piv)
    assert rounds >= 1


def test_device_pivot_selection_degenerate_inputs(rn):
    # no reverse neighbours at all: every vertex is a singleton pivot
    n = 300
    nplus = np.full((n, 4), -1, np.int32)
    offs, ids = oracle.reverse_knn(nplus, 2)
    got_of, npiv, _ = rn.select_pivots_gpu(dev(nplus), 2, dev(offs), dev(np.zeros(1, np.int32)))
    assert (host(got_of) == -1).all() and npiv == n
    # a star: vertex 0 is everyone's nearest
    nplus = np.full((n, 4), -1, np.int32)
    nplus[1:, 0] = 0
    nplus[0, 0] = 1
    offs, ids = oracle.reverse_knn(nplus, 1)
    want_of, _, _ = oracle.select_pivots(n, offs, ids)
    got_of, _, _ = rn.select_pivots_gpu(dev(nplus), 1, dev(offs), dev(ids))
    np.testing.assert_array_equal(host(got_of), want_of)


def test_merge_host_and_device_pivots_agree(rn):
    segs = [gen.gaussian(3000, 32, 81), gen.gaussian(2500, 32, 82)]
    gs = [oracle.build_graph(s, 16, 32, 1.2) for s in segs]
    tsegs = [(dev(s), dev(g), e) for s, (g, e) in zip(segs, gs)]
    a, sa = rn.merge(tsegs, rn.params(16, 32, 1.2))
    b, sb = rn.merge(tsegs, rn.params(16, 32, 1.2, flags=rn.FLAG_HOST_PIVOTS))
    np.testing.assert_array_equal(host(a), host(b))
    assert sa["pivots"] == sb["pivots"]


# ------------------------------------------- precision pattern (BF16 / FP8)

@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("kind,d,w,R", [
    ("gauss", 32, 64, 32), ("gauss", 128, 48, 32), ("deep", 96, 64, 32), ("sift", 128, 64, 32),
    ("embed", 256, 40, 32), ("gauss", 128, 100, 32),
    # pools of up to 128 raw candidates, K-chunked rows, the split BF16 tile (d >= 384)
    ("deep", 96, 128, 64), ("sift", 128, 120, 64), ("embed", 768, 128, 64),
    ("gauss", 512, 128, 64), ("embed", 384, 96, 48), ("gauss", 1024, 70, 32),
    ("sift", 160, 128, 16),
    # pools above 128 overflow to the FP32 general kernel
    ("embed", 768, 150, 64),
    # BF16 at L2 and d <= 128 with pools <= 64: two owners per tile (real-valued
    # rows need the lo term, integer rows do not); R = pool size; d = 16
    ("deepl2", 96, 64, 32), ("deepl2", 96, 40, 16), ("deepl2", 128, 64, 64),
    ("gauss", 16, 64, 32), ("gauss", 64, 33, 8), ("sift", 48, 64, 32),
    # integer rows spanning <= 256 (far from 0): hi terms only; spanning 510: hi and lo
    ("offset", 128, 64, 32), ("wide", 128, 64, 32)])
def test_low_precision_prune_equals_fp32(rn, prec, kind, d, w, R):
    n = 3000
    X = {"gauss": lambda: gen.gaussian(n, d, 90),
         "deep": lambda: gen.deep_like(n, 91, d=d),
         "deepl2": lambda: gen.deep_like(n, 94, d=d),
         "sift": lambda: gen.sift_like(n, 92, d=d),
         "offset": lambda: gen.sift_like(n, 92, d=d) + np.float32(1000.0),
         "wide": lambda: gen.sift_like(n, 92, d=d) * np.float32(2.0),
         "embed": lambda: gen.embed_like(n, 93, d=d, n_comp=50)}[kind]()
    metric = oracle.IP if kind in ("deep", "embed") else oracle.L2
    owners, pool = _pools(n, w, 7 * d + w, 800)
    Xd, od, pd_ = dev(X), dev(owners), dev(pool)
    want = rn.prune(Xd, od, pd_, R, 1.2, metric=metric)
    got = rn.prune(Xd, od, pd_, R, 1.2, metric=metric, prec=prec)
    np.testing.assert_array_equal(host(got), host(want))
    want2 = rn.prune(Xd, od, pd_, R, 1.2, metric=metric, keep_all_if_fit=True)
    got2 = rn.prune(Xd, od, pd_, R, 1.2, metric=metric, keep_all_if_fit=True, prec=prec)
    np.testing.assert_array_equal(host(got2), host(want2))


@pytest.mark.parametrize("prec", [1, 2])
def test_low_precision_merge_equals_fp32(rn, prec):
    for segs, metric in ((gen.tiny_case(n_per_seg=3000)[0], oracle.L2),
                         ([gen.sift_like(4000, 95, d=128), gen.sift_like(3000, 96, d=128)],
                          oracle.L2),
                         ([gen.deep_like(3000, 97, d=96), gen.deep_like(2500, 98, d=96)],
                          oracle.IP),
                         ([gen.deep_like(6000, 99, d=96), gen.deep_like(5000, 100, d=96)],
                          oracle.L2)):
        R, L = (16, 32) if segs[0].shape[1] == 32 else (32, 64)
        gs = [oracle.build_graph(s, R, L, 1.2, metric=metric) for s in segs]
        tsegs = [(dev(s), dev(g), e) for s, (g, e) in zip(segs, gs)]
        a, sa = rn.merge(tsegs, rn.params(R, L, 1.2, metric=metric))
        b, sb = rn.merge(tsegs, rn.params(R, L, 1.2, metric=metric, prec=prec))
        np.testing.assert_array_equal(host(b), host(a))
        assert sa["rechecks"] == 0
        # sampled tile distances stay inside their error bounds
        assert sb["tile_error"][3] > 0 and sb["tile_error"][2] <= 1.0
        assert sa["tile_error"][3] == 0
        if segs[0].dtype == np.float32 and not (segs[0] == np.rint(segs[0])).all():
            assert sb["rechecks"] > 0       # real-valued data: some decisions re-decided


@pytest.mark.parametrize("prec", [1, 2])
def test_low_precision_merge_equals_fp32_embedding_shape(rn, prec):
    # d = 768, inner product, R = 64, L = 128: source pools of R + c_cross = 128
    # candidates go to the tensor-core tile (the split BF16 tile for prec 1)
    X = gen.embed_like(4000, 99, d=768, n_comp=40)
    segs = [X[:2200], X[2200:]]
    gs = [oracle.build_graph(s, 64, 128, 1.2, metric=oracle.IP) for s in segs]
    tsegs = [(dev(s), dev(g), e) for s, (g, e) in zip(segs, gs)]
    a, _ = rn.merge(tsegs, rn.params(64, 128, 1.2, metric=oracle.IP))
    b, sb = rn.merge(tsegs, rn.params(64, 128, 1.2, metric=oracle.IP, prec=prec))
    np.testing.assert_array_equal(host(b), host(a))
    assert sb["rechecks"] > 0
    assert sb["tile_error"][3] > 0 and sb["tile_error"][2] <= 1.0


# ---------------------------------------------------------------- autotuner

def test_search_variants_and_autotuned_launch_agree(rn, monkeypatch):
    # 66k queries trigger the autotuner (16 chunks of the launch run with
    # different launch shapes, with and without the L2 prefetch); every variant
    # must give the same results as the oracle.
    X = gen.sift_like(20000, 101, d=32)
    adj, ep = oracle.build_graph(X, 16, 32, 1.2)
    Q = gen.sift_like(66000, 102, d=32)
    seeds = np.full((len(Q), 1), ep, np.int32)
    want, _, _, _, _ = oracle.beam_search(X, adj, Q, seeds, 24, 10)
    outs = []
    for force in ("0", "1", "2", "3", None):
        if force is None:
            monkeypatch.delenv("RNSM_SEARCH_VARIANT", raising=False)
        else:
            monkeypatch.setenv("RNSM_SEARCH_VARIANT", force)
        ids, _, _ = rn.search(dev(X), dev(adj), dev(Q), dev(seeds), 24, 10)
        outs.append(host(ids))
    for o in outs:
        np.testing.assert_array_equal(o, want)


def test_expand_autotuned_on_large_batch(rn):
    X = gen.sift_like(66000, 103, d=32)
    adj, _ = oracle.build_graph(X, 16, 32, 1.2)
    want, _, _, _ = oracle.expand(X, adj, 12)
    got = rn.expand(dev(X), dev(adj), 12)
    np.testing.assert_array_equal(host(got), want)


@pytest.mark.parametrize("kind", ["sift", "deepl2"])
def test_prune_variants_and_autotuned_choice_agree(rn, monkeypatch, kind):
    # the prune variants (pair tile, general tile, FP32 walk and triangle) take the
    # FP32 decisions; 250,000 owners trigger the autotuner (slices of the owners
    # run with each variant in turn), whose choice must not change the result
    n = 260000
    X = gen.sift_like(n, 111, d=128) if kind == "sift" else gen.deep_like(n, 112, d=96)
    owners, pool = _pools(n, 64, 113, 250000)
    Xd, od, pd_ = dev(X), dev(owners), dev(pool)
    ref = host(rn.prune(Xd, od, pd_, 32, 1.2))
    want, _ = oracle.prune(X, owners[:2000].astype(np.int64), pool[:2000], 32, 1.2)
    if kind == "sift":   # integer rows: exact against the oracle
        np.testing.assert_array_equal(ref[:2000], want)
    for prec in (rn.BF16, rn.FP8):
        for force in ("1", "2", "0", "3", None):
            if force is None:
                monkeypatch.delenv("RNSM_PRUNE_VARIANT", raising=False)
            else:
                monkeypatch.setenv("RNSM_PRUNE_VARIANT", force)
            got = host(rn.prune(Xd, od, pd_, 32, 1.2, prec=prec))
            np.testing.assert_array_equal(got, ref, err_msg=f"prec {prec} variant {force}")
        # the tuned choice, reused
        np.testing.assert_array_equal(host(rn.prune(Xd, od, pd_, 32, 1.2, prec=prec)), ref)
