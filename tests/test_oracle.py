"""Pins of the FP64 oracle against facts fixed outside it: hand-worked
examples (tests/golden), brute force, closed forms, exhaustive enumeration and
invariants stated by the paper.  CPU only."""
import itertools
import os

import numpy as np
import pytest

import oracle
from workloads import generators as gen

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _lines(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]


def _np_dist(X, q, metric):
    X = X.astype(np.float64)
    q = q.astype(np.float64)
    if metric == oracle.L2:
        return ((X - q) ** 2).sum(axis=1)
    return 1.0 - X @ q


def _np_topk(X, q, k, metric):
    d = _np_dist(X, q, metric)
    order = np.lexsort((np.arange(len(d)), d))
    return order[:k], d[order[:k]]


# ---------------------------------------------------------------- distances

def test_distance_hand_values():
    a = np.array([1, 2, 3, 4], np.float32)
    b = np.array([4, 6, 3, 0], np.float32)
    assert oracle.distance(a, b, oracle.L2) == 9 + 16 + 0 + 16
    assert oracle.distance(a, b, oracle.IP) == 1 - (4 + 12 + 9 + 0)


def test_distance_unit_norm_l2_is_twice_ip():
    # For unit vectors ||x-y||^2 = 2 - 2<x,y> = 2 * (1 - <x,y>).
    X = gen.deep_like(64, seed=11, d=96)
    for i in range(0, 64, 2):
        l2 = oracle.distance(X[i], X[i + 1], oracle.L2)
        ip = oracle.distance(X[i], X[i + 1], oracle.IP)
        assert abs(l2 - 2 * ip) < 1e-6


# -------------------------------------------------------------- brute force

@pytest.mark.parametrize("metric", [oracle.L2, oracle.IP])
def test_bruteforce_matches_library_sort(metric):
    X = gen.deep_like(700, seed=3, d=24)
    Q = gen.deep_like(20, seed=4, d=24)
    ids, dd = oracle.bruteforce_knn(X, Q, 13, metric)
    for qi in range(len(Q)):
        ref_ids, ref_d = _np_topk(X, Q[qi], 13, metric)
        np.testing.assert_array_equal(ids[qi], ref_ids)
        np.testing.assert_allclose(dd[qi], ref_d, rtol=1e-12, atol=1e-12)


# ------------------------------------------------------------- beam search

def test_beam_search_golden_trap():
    X = np.array([[0.0], [-1.0], [10.0]], np.float32)
    adj = np.array([[1], [2], [1]], np.int32)
    q = np.array([[9.0]], np.float32)
    for ef, res, ndc, nexp in _lines("beam_search_trap.txt"):
        ef = int(ef)
        want = [int(x) for x in res.split(",")]
        ids, _, nd, ne, _ = oracle.beam_search(X, adj, q, [[0]], ef, ef)
        assert list(ids[0][: len(want)]) == want
        assert nd[0] == int(ndc) and ne[0] == int(nexp)


@pytest.mark.parametrize("metric", [oracle.L2, oracle.IP])
def test_beam_search_complete_graph_is_exact(metric):
    # Complete graph: expanding the seed evaluates every vertex once, so the
    # final C is the exact top-ef; NDC = n, and every final entry is expanded
    # plus the seed itself if it fell out of C: min(ef, n) + [seed not kept].
    n, d = 60, 8
    X = gen.deep_like(n, seed=5, d=d)
    adj = np.array([[j for j in range(n) if j != i] for i in range(n)], np.int32)
    Q = gen.deep_like(7, seed=6, d=d)
    for ef in (1, 5, 17, 60):
        ids, dd, ndc, nexp, _ = oracle.beam_search(X, adj, Q, [[3]], ef, ef, metric)
        for qi in range(len(Q)):
            ref, _ = _np_topk(X, Q[qi], ef, metric)
            np.testing.assert_array_equal(ids[qi], ref)
            assert nexp[qi] == min(ef, n) + (3 not in ref)
        assert (ndc == n).all()


def _reachable(adj, src):
    seen = {src}
    stack = [src]
    while stack:
        u = stack.pop()
        for v in adj[u]:
            if v >= 0 and v not in seen:
                seen.add(int(v))
                stack.append(int(v))
    return np.array(sorted(seen))


def test_beam_search_ef_ge_n_equals_bruteforce_on_reachable_set():
    # With ef >= n nothing is ever evicted, so the search evaluates exactly the
    # vertices reachable from the entry: result = their brute-force order.
    X = gen.gaussian(200, 6, seed=7)
    adj, ep = oracle.build_graph(X, 8, 16, 1.2)
    reach = _reachable(adj, ep)
    Q = gen.gaussian(10, 6, seed=8)
    ids, _, ndc, _, _ = oracle.beam_search(X, adj, Q, [[ep]], 200, 200)
    for qi in range(len(Q)):
        ref, _ = _np_topk(X[reach], Q[qi], len(reach), oracle.L2)
        np.testing.assert_array_equal(ids[qi][: len(reach)], reach[ref])
        assert (ids[qi][len(reach):] == -1).all()
    assert (ndc == len(reach)).all()


def test_beam_search_results_sorted_unique_and_seed_dedupe():
    X = gen.gaussian(500, 16, seed=9)
    adj, ep = oracle.build_graph(X, 12, 24, 1.2)
    Q = gen.gaussian(30, 16, seed=10)
    seeds = np.tile(np.array([[ep, ep, -1, 7, 7]], np.int32), (30, 1))
    ids, dd, _, _, _ = oracle.beam_search(X, adj, Q, seeds, 32, 32)
    for qi in range(30):
        assert len(set(ids[qi])) == 32
        assert np.all(np.diff(dd[qi]) >= 0)
        np.testing.assert_allclose(dd[qi], _np_dist(X[ids[qi]], Q[qi], oracle.L2), rtol=1e-12)


# ------------------------------------------------------------------- prune

def test_prune_golden_line():
    for alpha, R, cands, kept in _lines("prune_line.txt"):
        cs = [float(x) for x in cands.split(";")]
        want = [float(x) for x in kept.split(";")]
        X = np.array([[0.0]] + [[c] for c in cs], np.float32)
        W = np.arange(1, len(cs) + 1, dtype=np.int32)[None, :]
        out, _ = oracle.prune(X, [0], W, int(R), float(alpha))
        got = [float(X[i, 0]) for i in out[0] if i >= 0]
        assert got == want, (alpha, R, cands)


def _prune_case(seed, n=40, d=5):
    X = gen.gaussian(n, d, seed)
    W = np.arange(1, n, dtype=np.int32)[None, :]
    return X, W


def test_prune_special_cases_alpha_zero_and_huge():
    X, W = _prune_case(21)
    order, _ = _np_topk(X[1:], X[0], 39, oracle.L2)
    out0, _ = oracle.prune(X, [0], W, 10, 0.0)
    assert list(out0[0][:1]) == [order[0] + 1] and (out0[0][1:] == -1).all()
    outH, _ = oracle.prune(X, [0], W, 10, 1e30)
    np.testing.assert_array_equal(outH[0], order[:10] + 1)


@pytest.mark.parametrize("seed", range(5))
@pytest.mark.parametrize("alpha", [1.0, 1.2, 2.0])
def test_prune_invariants_and_maximality(seed, alpha):
    # Kept list: subset of W, sorted by distance, nearest always kept, every
    # kept pair passes the rule, and every candidate skipped before the R-th
    # keep is occluded by a kept one that precedes it.
    X, W = _prune_case(100 + seed)
    R = 6
    out, _ = oracle.prune(X, [0], W, R, alpha)
    kept = [i for i in out[0] if i >= 0]
    d0 = _np_dist(X, X[0], oracle.L2)
    order = [int(i) for i in np.lexsort((np.arange(len(d0)), d0)) if i != 0]
    assert kept[0] == order[0]
    assert all(d0[a] <= d0[b] for a, b in zip(kept, kept[1:]))
    a32 = float(np.float32(alpha))
    for i, c in enumerate(kept):
        for s in kept[:i]:
            assert not (a32 * _np_dist(X[[s]], X[c], oracle.L2)[0] <= d0[c])
    last = order.index(kept[-1])
    for c in order[:last]:
        if c in kept:
            continue
        prev = [s for s in kept if order.index(s) < order.index(c)]
        assert any(a32 * _np_dist(X[[s]], X[c], oracle.L2)[0] <= d0[c] for s in prev)
    if len(kept) < R:  # stopped because W ran out: every later one occluded
        for c in order[last + 1:]:
            assert any(a32 * _np_dist(X[[s]], X[c], oracle.L2)[0] <= d0[c] for s in kept)


def test_prune_drops_owner_duplicates_and_padding():
    X, _ = _prune_case(5)
    W = np.array([[0, 3, 3, -1, 5, 0, 5, 7]], np.int32)
    out, _ = oracle.prune(X, [0], W, 8, 1e30)
    kept = [i for i in out[0] if i >= 0]
    assert sorted(kept) == [3, 5, 7]


def test_prune_keep_all_if_fit():
    X, _ = _prune_case(6)
    W = np.array([[4, 2, 9]], np.int32)
    out, _ = oracle.prune(X, [0], W, 3, 0.0, keep_all_if_fit=True)
    d0 = _np_dist(X, X[0], oracle.L2)
    assert list(out[0]) == sorted([4, 2, 9], key=lambda i: (d0[i], i))


# -------------------------------------------------- reverse kNN and pivots

def test_reverse_knn_is_transpose_of_knn_lists():
    rng = np.random.default_rng(0)
    n, kp, k = 300, 8, 3
    nplus = np.array([rng.choice([j for j in range(n) if j != i], kp, replace=False)
                      for i in range(n)], np.int32)
    offs, ids = oracle.reverse_knn(nplus, k)
    assert offs[-1] == n * k
    for x in range(n):
        want = sorted(int(y) for y in np.nonzero((nplus[:, :k] == x).any(axis=1))[0])
        assert list(ids[offs[x]:offs[x + 1]]) == want


def _naive_greedy(n, offs, ids):
    """Plain greedy: repeatedly select the uncovered x of largest current gain
    |R_k(x) \\ Covered| (ties: lower id).  Lazy evaluation in Algorithm 2 is
    an implementation of exactly this rule."""
    covered = np.zeros(n, bool)
    piv_of = np.full(n, -2, np.int64)
    order = []
    while not covered.all():
        best, bg = -1, -1
        for x in range(n):
            if covered[x]:
                continue
            g = int((~covered[ids[offs[x]:offs[x + 1]]]).sum())
            if g > bg:
                best, bg = x, g
        for y in ids[offs[best]:offs[best + 1]]:
            if not covered[y]:
                covered[y] = True
                piv_of[y] = best
        covered[best] = True
        piv_of[best] = -1
        order.append(best)
    return piv_of, order


@pytest.mark.parametrize("seed", range(4))
def test_lazy_greedy_equals_plain_greedy(seed):
    X = gen.gaussian(250, 6, 30 + seed)
    adj, _ = oracle.build_graph(X, 8, 16, 1.2)
    nplus, _, _, _ = oracle.expand(X, adj, 10)
    offs, ids = oracle.reverse_knn(nplus, 4)
    piv_of, piv, dep = oracle.select_pivots(250, offs, ids)
    ref_of, ref_order = _naive_greedy(250, offs, ids)
    np.testing.assert_array_equal(piv_of, ref_of)
    assert list(piv) == ref_order
    # Every vertex is a pivot or a follower (U is empty, Section 4.2) and each
    # follower y has its pivot among its k nearest (p in N_k(y)).
    assert (piv_of >= -1).all()
    for y in range(250):
        if piv_of[y] >= 0:
            assert piv_of[y] in nplus[y, :4]


def test_pivot_golden_star():
    # Worked by hand (Algorithm 2, Phase 2), k = 1 (first column of N+):
    # R_1(0) = {1,2,3,4} (a hub of gain 4), R_1(1) = {0}, R_1(5) = {6},
    # R_1(6) = {5}.  Pop 0 (gain 4): pivot, covers 0..4.  Pop 1: covered,
    # skipped.  5 and 6 tie at gain 1: the lower id 5 is the pivot of 6.
    nplus = np.array([[1, 2], [0, 2], [0, 1], [0, 1], [0, 3], [6, 0], [5, 0]], np.int32)
    offs, ids = oracle.reverse_knn(nplus, 1)
    piv_of, piv, dep = oracle.select_pivots(7, offs, ids)
    assert list(piv) == [0, 5]
    assert list(piv_of) == [-1, 0, 0, 0, 0, -1, 5]
    assert dep == 0


def test_idps_cost_reduction_identity():
    # Theorem (IDPS NP-hard) proof: with delta = 1 between distinct nodes,
    # gamma = 2 and beta = 1, any independent dominating set P costs |P| + |V|.
    rng = np.random.default_rng(1)
    n = 9
    A = np.zeros((n, n), np.uint8)
    for _ in range(14):
        a, b = rng.integers(0, n, 2)
        if a != b:
            A[a, b] = A[b, a] = 1
    D = 1.0 - np.eye(n)
    found = 0
    for mask in range(1, 1 << n):
        P = np.array([(mask >> i) & 1 for i in range(n)], np.uint8)
        idx = np.nonzero(P)[0]
        if any(A[a, b] for a in idx for b in idx):
            continue
        if not all(P[v] or A[v, idx].any() for v in range(n)):
            continue
        found += 1
        assert oracle.idps_cost(D, A, P, 2.0, 1.0) == len(idx) + n
    assert found > 0


# ------------------------------------------------------------------- MOS

def _diameter(m, edges):
    INF = 10 ** 9
    H = np.full((m, m), INF)
    np.fill_diagonal(H, 0)
    for a, b in edges:
        H[a, b] = H[b, a] = 1
    for k in range(m):
        H = np.minimum(H, H[:, [k]] + H[[k], :])
    return H.max()


def _exhaustive_opt(C, Rm, Delta):
    m = C.shape[0]
    pairs = list(itertools.combinations(range(m), 2))
    best = np.inf
    for mask in range(1 << len(pairs)):
        E = [pairs[i] for i in range(len(pairs)) if (mask >> i) & 1]
        deg = np.zeros(m, int)
        for a, b in E:
            deg[a] += 1
            deg[b] += 1
        if (deg > Rm).any():
            continue
        if _diameter(m, E) > Delta:
            continue
        best = min(best, sum(C[a, b] for a, b in E))
    return best


@pytest.mark.parametrize("seed", range(6))
def test_mos_feasible_and_bounded_by_exhaustive_optimum(seed):
    rng = np.random.default_rng(seed)
    m = 4 + seed % 3            # 4..6 segments: at most 2^15 edge subsets
    cen = rng.standard_normal((m, 3))
    C = np.sqrt(((cen[:, None] - cen[None]) ** 2).sum(-1))
    Rm = int(np.ceil(np.sqrt(m - 1))) + 1
    edges, flags = oracle.mos(C, Rm, 2)
    opt = _exhaustive_opt(C, Rm, 2)
    cost = sum(C[a, b] for a, b in edges)
    assert _diameter(m, edges) <= 2                 # connected, diameter <= Delta
    assert len(set(tuple(sorted(e)) for e in edges)) == len(edges)
    if not flags.any():
        deg = np.bincount(np.array(edges).ravel(), minlength=m)
        assert deg.max() <= Rm
        assert cost >= opt - 1e-12                      # optimum is a lower bound
    assert np.isfinite(opt)


def test_mos_two_segments_single_edge_and_orientation():
    plan = oracle.mos_plan([100, 300])
    assert plan == [(0, 1, 1.0)]
    plan = oracle.mos_plan([300, 300])
    assert [(a, b) for a, b, _ in plan] == [(1, 0)]


def test_mos_plan_order_and_orientation():
    rng = np.random.default_rng(5)
    m = 8
    cen = rng.standard_normal((m, 4)).astype(np.float32)
    sizes = rng.integers(10, 1000, m)
    plan = oracle.mos_plan(sizes, cen)
    costs = [c for _, _, c in plan]
    assert costs == sorted(costs)
    for s, t, c in plan:
        assert sizes[s] <= sizes[t]
        assert abs(c - np.linalg.norm(cen[s].astype(np.float64) - cen[t])) < 1e-9
    assert _diameter(m, [(s, t) for s, t, _ in plan]) <= 2


def test_mos_unit_cost_complete_when_bound_allows():
    # With Rm >= m-1 every vertex may reach every other directly; the greedy
    # adds edges only while some pair is more than Delta hops apart.
    edges, flags = oracle.mos(1.0 - np.eye(3), 2, 2)
    assert len(edges) == 2 and not flags.any()    # a path of 3 has diameter 2


# ------------------------------------------------------ builder and merge

def _graph_invariants(adj, R, n_total, self_ids=None):
    assert adj.shape[1] == R
    assert ((adj >= -1) & (adj < n_total)).all()
    for v in range(adj.shape[0]):
        row = [int(u) for u in adj[v] if u >= 0]
        assert len(row) == len(set(row))
        me = v if self_ids is None else self_ids[v]
        assert me not in row
        # -1 padding only at the end
        k = len(row)
        assert (adj[v, :k] >= 0).all() and (adj[v, k:] == -1).all()


def test_build_invariants_and_quality():
    X = gen.gaussian(1500, 16, 40)
    adj, ep = oracle.build_graph(X, 12, 24, 1.2)
    _graph_invariants(adj, 12, 1500)
    assert ep == oracle.medoid(X)
    Q = gen.gaussian(100, 16, 41)
    _, gd = oracle.bruteforce_knn(X, Q, 10)
    ids, _, _, _, _ = oracle.beam_search(X, adj, Q, [[ep]], 64, 10)
    assert oracle.recall_at_k(ids, X, gd, Q) > 0.9


def test_medoid_closed_form():
    # Symmetric 1-D set: the centroid is 0 and the vertex at 0 is nearest.
    X = np.array([[-3.0], [5.0], [0.0], [-5.0], [3.0]], np.float32)
    assert oracle.medoid(X) == 2


def _tiny_merge_inputs(n=600, d=8, R=8, L=16, seed=50):
    segs = [gen.gaussian(n, d, seed), gen.gaussian(n // 2, d, seed + 1)]
    gs = [oracle.build_graph(s, R, L, 1.2) for s in segs]
    return segs, [g for g, _ in gs], [e for _, e in gs]


def test_merge_invariants_and_stats():
    segs, graphs, entries = _tiny_merge_inputs()
    plan = oracle.pair_plan([len(s) for s in segs])
    assert plan == [(1, 0)]
    out, st = oracle.rnsm_merge(segs, graphs, entries, plan, 8, 16, 1.2)
    N = sum(len(s) for s in segs)
    _graph_invariants(out, 8, N)
    assert st["pivots"] + st["followers"] == len(segs[1])
    n0 = len(segs[0])
    # every source vertex got at least one cross edge candidate considered;
    # target vertices gain cross edges only through reverse edges.
    cross_src = (out[n0:] < n0) & (out[n0:] >= 0)
    assert cross_src.any(axis=1).mean() > 0.5
    rev = ((out[:n0] >= n0)).sum()
    assert 0 < rev <= st["reverse_edges"]


def test_merge_reduces_to_exact_topk_when_search_is_exhaustive():
    # With complete target graphs and ef >= n_t every search (naive or
    # sliding) returns the exact top-ef, so each source list must equal
    # prune(list(v) u exact top-c_cross of the target) -- brute force + the
    # prune pinned above.
    n, d, R = 40, 4, 6
    nt = R + 1
    tgt = gen.gaussian(nt, d, 62)
    tgraph = np.array([[j for j in range(nt) if j != i] for i in range(nt)], np.int32)
    src = gen.gaussian(n, d, 60)
    sgraph, sep = oracle.build_graph(src, R, 12, 1.2)
    L = nt + 2
    out, _ = oracle.rnsm_merge([tgt, src], [tgraph, sgraph], [0, sep], [(1, 0)], R, L, 1.2,
                               ef_slide=L, c_cross=L)
    X = np.concatenate([tgt, src])
    for v in range(n):
        top, _ = _np_topk(tgt, src[v], nt, oracle.L2)
        own = np.where(sgraph[v] >= 0, sgraph[v] + nt, -1)
        pool = np.concatenate([own, top]).astype(np.int32)[None, :]
        want, _ = oracle.prune(X, [nt + v], pool, R, 1.2)
        np.testing.assert_array_equal(out[nt + v], want[0])


def test_merge_single_segment_is_identity():
    X = gen.gaussian(300, 8, 70)
    adj, ep = oracle.build_graph(X, 8, 16, 1.2)
    out, _ = oracle.rnsm_merge([X], [adj], [ep], [], 8, 16, 1.2)
    np.testing.assert_array_equal(out, adj)


def test_merge_quality_comparable_to_rebuild():
    # Section 6 Exp-1: the merged graph searches about as well as a rebuild.
    segs, Q = gen.tiny_case(n_per_seg=1500, d=16, nq=200)
    gs = [oracle.build_graph(s, 12, 24, 1.2) for s in segs]
    out, st = oracle.rnsm_merge(segs, [g for g, _ in gs], [e for _, e in gs],
                                oracle.pair_plan([1500, 1500]), 12, 24, 1.2)
    X = np.concatenate(segs)
    _, gd = oracle.bruteforce_knn(X, Q, 10)
    reb, rep = oracle.build_graph(X, 12, 24, 1.2)
    ids_m, _, _, _, _ = oracle.beam_search(X, out, Q, [[gs[0][1]]], 32, 10)
    ids_r, _, _, _, _ = oracle.beam_search(X, reb, Q, [[rep]], 32, 10)
    rm = oracle.recall_at_k(ids_m, X, gd, Q)
    rr = oracle.recall_at_k(ids_r, X, gd, Q)
    assert rm > rr - 0.05, (rm, rr)
    # pivots are a minority (about 20% in the paper's complexity analysis)
    assert 0.05 < st["pivots"] / 1500 < 0.45


def test_oracle_deterministic_across_thread_counts():
    segs, graphs, entries = _tiny_merge_inputs(n=400)
    a, _ = oracle.rnsm_merge(segs, graphs, entries, [(1, 0)], 8, 16, 1.2, threads=1)
    b, _ = oracle.rnsm_merge(segs, graphs, entries, [(1, 0)], 8, 16, 1.2, threads=4)
    np.testing.assert_array_equal(a, b)


# ------------------------------------------- hand-worked pins (tests/golden)

def _read_blocks(name):
    """Lines of a golden file grouped into blocks ending with 'end'."""
    blocks, cur = [], []
    for parts in _lines(name):
        if parts[0] == "end":
            blocks.append(cur)
            cur = []
        else:
            cur.append(parts)
    if cur:
        blocks.append(cur)
    return blocks


def test_mos_golden_trace():
    # Algorithm 3, traced by hand: exact edge list (insertion order) and the
    # degree-bound flags, including the cheapest vertex beyond Delta hops, a
    # relay on either saturated end, the no-relay and both-saturated fallbacks
    # and the tie rules.
    blocks = _read_blocks("mos_trace.txt")
    assert len(blocks) == 3
    for blk in blocks:
        C = np.array([[float(x) for x in p[1].split(",")] for p in blk if p[0] == "C"])
        (rl,) = [p for p in blk if p[0] == "R"]
        Rm, Delta = int(rl[1]), int(rl[3])
        (el,) = [p for p in blk if p[0] == "E"]
        want = [tuple(int(t) for t in e.split(",")) for e in el[1:]]
        edges, flags = oracle.mos(C, Rm, Delta)
        assert edges == [(a, b) for a, b, _ in want]
        assert list(flags.astype(int)) == [f for _, _, f in want]
        assert _diameter(C.shape[0], edges) <= Delta


def test_reverse_edges_golden_line():
    rows = _lines("reverse_edges_line.txt")
    X = np.array([[float(x)] for x in rows[0][1].split(",")], np.float32)
    (pl,) = [p for p in rows if p[0] == "P"]
    R, alpha = int(pl[1]), float(pl[2])
    lists = np.full((len(X), R), -1, np.int32)
    for p in rows:
        if p[0] == "L":
            lists[int(p[1])] = [int(t) for t in p[2].split(",")]
    eu = [int(p[1]) for p in rows if p[0] == "E"]
    ev = [int(p[2]) for p in rows if p[0] == "E"]
    want = lists.copy()
    for p in rows:
        if p[0] == "W":
            want[int(p[1])] = [int(t) for t in p[2].split(",")]
    got = oracle.reverse_edges(X, lists, eu, ev, alpha)
    np.testing.assert_array_equal(got, want)
    # The edge order does not matter (the pools are sets).
    perm = np.random.default_rng(3).permutation(len(eu))
    got2 = oracle.reverse_edges(X, lists, np.array(eu)[perm], np.array(ev)[perm], alpha)
    np.testing.assert_array_equal(got2, want)


def test_expand_golden_duplicates_and_evicted_seed():
    X = np.array([[5.0], [5.0], [5.0], [9.0], [0.0]], np.float32)
    n = len(X)
    adj = np.array([[j for j in range(n) if j != i] for i in range(n)], np.int32)
    for kp, rows in _lines("expand_duplicates.txt"):
        want = np.array([[int(t) for t in r.split(",")] for r in rows.split(";")], np.int32)
        got, _, _, _ = oracle.expand(X, adj, int(kp))
        np.testing.assert_array_equal(got, want)


@pytest.mark.parametrize("metric", [oracle.L2, oracle.IP])
@pytest.mark.parametrize("k_plus", [1, 4, 15])
def test_expand_complete_graph_is_bruteforce_without_self(metric, k_plus):
    # On a complete graph the search seeded at v evaluates every vertex, so
    # N+(v) is exactly the k+ nearest other vertices (no distance ties here).
    n, d = 50, 6
    X = gen.deep_like(n, seed=90 + k_plus, d=d)
    adj = np.array([[j for j in range(n) if j != i] for i in range(n)], np.int32)
    got, ndc, _, _ = oracle.expand(X, adj, k_plus, metric)
    for v in range(n):
        dist = _np_dist(X, X[v], metric)
        dist[v] = np.inf
        ref = np.lexsort((np.arange(n), dist))[:k_plus]
        np.testing.assert_array_equal(got[v], ref)
    assert (ndc == n).all()


def test_recall_golden_ties():
    rows = _lines("recall_ties.txt")
    X = np.array([[float(x)] for x in rows[0][1].split(",")], np.float32)
    Q = np.array([[float(x)] for x in rows[1][1].split(",")], np.float32)
    gt = np.array([[float(x) for x in p[1].split(",")] for p in rows if p[0] == "G"])
    assert gt.shape == (2, 11)
    for case, q0, q1, want in (p for p in rows if p[0] in "abcd"):
        found = np.array([[int(t) for t in q0.split(",")], [int(t) for t in q1.split(",")]])
        assert oracle.recall_at_k(found, X, gt, Q, k=10) == pytest.approx(float(want)), case


def _cm_by_parts(segs, graphs, entries, plan, R, L, alpha, c_cross):
    """Cross-query Merge (Section 3.1), composed from the pinned parts: for
    each plan edge s -> t in order, every source vertex runs a naive beam
    search of the frozen target graph from its entry (ef = L); its pool is its
    current list and the first c_cross results; the pool is pruned; kept
    cross edges add reverse edges into t."""
    X = np.concatenate(segs)
    off = np.concatenate([[0], np.cumsum([len(s) for s in segs])])
    lists = np.full((len(X), R), -1, np.int32)
    for s, g in enumerate(graphs):
        r = g.shape[1]
        lists[off[s]:off[s + 1], :r] = np.where(g >= 0, g + off[s], -1)
    for s, t in plan:
        Q = segs[s]
        seeds = np.full((len(Q), 1), entries[t], np.int32)
        res, _, _, _, _ = oracle.beam_search(segs[t], graphs[t], Q, seeds, L, L)
        cross = np.where(res[:, :c_cross] >= 0, res[:, :c_cross] + off[t], -1)
        owners = np.arange(off[s], off[s + 1], dtype=np.int64)
        pool = np.concatenate([lists[off[s]:off[s + 1]], cross], axis=1).astype(np.int32)
        new, _ = oracle.prune(X, owners, pool, R, alpha)
        lists[off[s]:off[s + 1]] = new
        eu, ev = [], []
        for i, v in enumerate(owners):
            for u in new[i]:
                if off[t] <= u < off[t + 1]:
                    eu.append(u)
                    ev.append(v)
        lists = oracle.reverse_edges(X, lists, np.array(eu, np.int32), np.array(ev, np.int32),
                                     alpha)
    return lists


def test_cm_merge_equals_its_pinned_parts():
    segs = [gen.gaussian(500, 8, 110), gen.gaussian(300, 8, 111), gen.gaussian(200, 8, 112)]
    gs = [oracle.build_graph(s, 8, 16, 1.2) for s in segs]
    graphs, entries = [g for g, _ in gs], [e for _, e in gs]
    for plan in ([(1, 0)], [(2, 0), (1, 0), (2, 1)]):
        got, st = oracle.rnsm_merge(segs, graphs, entries, plan, 8, 16, 1.2, cm=True)
        want = _cm_by_parts(segs, graphs, entries, plan, 8, 16, 1.2, c_cross=8)
        np.testing.assert_array_equal(got, want)
        assert st["followers"] == 0 and st["ndc_expand"] == 0
        assert st["pivots"] == sum(len(segs[s]) for s, _ in plan)
    # RNSM's followers slide from their pivot's results instead: a different graph
    rn_out, rst = oracle.rnsm_merge(segs, graphs, entries, [(1, 0)], 8, 16, 1.2)
    assert rst["followers"] > 0
    assert not np.array_equal(rn_out, oracle.rnsm_merge(segs, graphs, entries, [(1, 0)], 8, 16,
                                                         1.2, cm=True)[0])


def _union_cm_by_parts(segs, graphs, entries, plan, R, L, alpha, c_cross):
    """The multi-pair union variant with CM searches, from the pinned parts:
    every source vertex searches the frozen graph of each target of its plan
    edges (naive beam search from the target's entry, ef = L); one prune per
    source vertex over its list and the first c_cross results of each edge
    (blocks in plan order); then one reverse-edge pass over the kept edges
    into targets of the vertex's own plan edges."""
    X = np.concatenate(segs)
    off = np.concatenate([[0], np.cumsum([len(s) for s in segs])])
    lists = np.full((len(X), R), -1, np.int32)
    for s, g in enumerate(graphs):
        lists[off[s]:off[s + 1], :g.shape[1]] = np.where(g >= 0, g + off[s], -1)
    blocks = {}
    for s, t in plan:
        seeds = np.full((len(segs[s]), 1), entries[t], np.int32)
        res, _, _, _, _ = oracle.beam_search(segs[t], graphs[t], segs[s], seeds, L, L)
        blocks.setdefault(s, []).append(np.where(res[:, :c_cross] >= 0,
                                                 res[:, :c_cross] + off[t], -1))
    eu, ev = [], []
    for s in dict.fromkeys(s for s, _ in plan):
        owners = np.arange(off[s], off[s + 1], dtype=np.int64)
        pool = np.concatenate([lists[off[s]:off[s + 1]]] + blocks[s], axis=1).astype(np.int32)
        new, _ = oracle.prune(X, owners, pool, R, alpha)
        lists[off[s]:off[s + 1]] = new
        tgts = {t for s2, t in plan if s2 == s}
        seg_of = np.searchsorted(off, np.arange(len(X)), side="right") - 1
        for i, v in enumerate(owners):
            for u in new[i]:
                if u >= 0 and seg_of[u] in tgts:
                    eu.append(u)
                    ev.append(v)
    return oracle.reverse_edges(X, lists, np.array(eu, np.int32), np.array(ev, np.int32), alpha)


def test_union_prune_equals_its_pinned_parts():
    # with CM searches the union variant is a composition of pinned parts; the
    # plan has a source with three edges, a segment that is source and target,
    # and a target reached from two sources
    segs = [gen.gaussian(400, 8, 140), gen.gaussian(250, 8, 141), gen.gaussian(200, 8, 142),
            gen.gaussian(150, 8, 143)]
    gs = [oracle.build_graph(s, 8, 16, 1.2) for s in segs]
    graphs, entries = [g for g, _ in gs], [e for _, e in gs]
    plan = [(3, 0), (1, 0), (3, 2), (2, 0), (3, 1)]
    got, st = oracle.rnsm_merge(segs, graphs, entries, plan, 8, 16, 1.2, cm=True,
                                union_prune=True)
    want = _union_cm_by_parts(segs, graphs, entries, plan, 8, 16, 1.2, c_cross=8)
    np.testing.assert_array_equal(got, want)
    # it is not the edge-by-edge merge
    seq, _ = oracle.rnsm_merge(segs, graphs, entries, plan, 8, 16, 1.2, cm=True)
    assert not np.array_equal(got, seq)


def test_union_prune_with_one_edge_per_disjoint_pair_is_the_pairwise_merge():
    # each source one edge, no segment both source and target, distinct
    # targets: one prune per vertex and one reverse pass are the pairwise merges
    segs = [gen.gaussian(300, 8, 150), gen.gaussian(200, 8, 151), gen.gaussian(260, 8, 152),
            gen.gaussian(180, 8, 153)]
    gs = [oracle.build_graph(s, 8, 16, 1.2) for s in segs]
    graphs, entries = [g for g, _ in gs], [e for _, e in gs]
    plan = [(1, 0), (3, 2)]
    a, sa = oracle.rnsm_merge(segs, graphs, entries, plan, 8, 16, 1.2, union_prune=True)
    b, sb = oracle.rnsm_merge(segs, graphs, entries, plan, 8, 16, 1.2)
    np.testing.assert_array_equal(a, b)
    assert sa == sb
