"""FP64 CPU oracle of the RNSM merge path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its Python binding) never imports, links or executes anything here, and the
oracle shares no code with it.

The arithmetic lives in ``rnsm_oracle.c`` (plain C, FP64, OpenMP over
independent queries).  This module compiles it with gcc and wraps it with
numpy arrays.  See that file's header for the paper passages each function
follows.

Parity status: beam search, prune, reverse edges, neighbour expansion,
reverse-kNN inversion, pivot selection, IDPS cost, MOS, recall@k and
brute-force kNN are pinned by tests against hand-worked examples
(tests/golden), brute force, exhaustive restatements, closed forms and
invariants.  The end-to-end merge is pinned only by its parts, its invariants
and the recall tolerance ("parity unpinned" by the paper for the merge as a
whole).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rnsm_oracle.c")
_LIB = os.path.join(_HERE, "_build", "librnsm_oracle.so")
_lock = threading.Lock()
_lib = None

L2 = 0
IP = 1


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no -march, no fp contraction: identical
    results on x86_64 and aarch64)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-Wall", "-Wno-unknown-pragmas", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = C.CDLL(_LIB)
            _declare(lib)
            _lib = lib
    return _lib


P = C.c_void_p
i32, i64, f32, f64 = C.c_int32, C.c_int64, C.c_float, C.c_double


def _declare(lib):
    sig = {
        "orc_distance": (f64, [P, P, i64, i32]),
        "orc_max_threads": (i32, []),
        "orc_beam_search_batch": (i32, [P, i64, i64, P, i32, i32, P, i64, P, i32, i32, i32,
                                        P, P, P, P, P, i32]),
        "orc_medoid": (i32, [P, i64, i64, i32]),
        "orc_prune_batch": (i32, [P, i64, i32, P, i64, P, i32, i32, f32, i32, P, P, i32]),
        "orc_reverse_edges": (i32, [P, i64, i32, P, i32, P, P, i64, f32, i32]),
        "orc_expand": (i32, [P, i64, i64, P, i32, i32, i32, P, P, P, P, i32]),
        "orc_reverse_knn": (i32, [P, i64, i32, i32, P, P]),
        "orc_select_pivots": (i32, [i64, P, P, P, P, P, P]),
        "orc_idps_cost": (f64, [i64, P, P, P, f64, f64]),
        "orc_build": (i32, [P, i64, i64, i32, i32, i32, f32, i64, P, P, i32]),
        "orc_bruteforce_knn": (i32, [P, i64, i64, i32, P, i64, i32, P, P, i32]),
        "orc_rnsm_merge": (i32, [P, i64, P, i32, P, i32, P, i32, i32, i32, f32, i32, i32, i32,
                                 i32, P, P, i32, P, P, i32, i32, i32]),
        "orc_mos": (i32, [i32, P, i32, i32, P, P, P, P, i32]),
        "orc_mos_plan": (i32, [i32, P, P, i32, i32, i32, P, P, P, P, i32]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with status {rc}")


def max_threads() -> int:
    return int(_load().orc_max_threads())


def distance(a, b, metric=L2) -> float:
    a, b = _f32(a), _f32(b)
    return float(_load().orc_distance(_p(a), _p(b), a.shape[-1], metric))


def beam_search(X, adj, Q, seeds, ef, k, metric=L2, threads=0):
    """Algorithm 1 for every query.  seeds: [nq, n_seeds] (-1 = none).
    Returns ids [nq,k], dists [nq,k] (FP64), ndc [nq], expansions [nq], margin [nq]."""
    X, adj, Q = _f32(X), _i32(adj), _f32(Q)
    seeds = _i32(np.atleast_2d(seeds))
    nq = Q.shape[0]
    if seeds.shape[0] != nq:
        seeds = np.ascontiguousarray(np.broadcast_to(seeds, (nq, seeds.shape[1])), dtype=np.int32)
    ids = np.empty((nq, k), np.int32)
    dd = np.empty((nq, k), np.float64)
    ndc = np.empty(nq, np.int64)
    nexp = np.empty(nq, np.int64)
    mg = np.empty(nq, np.float64)
    rc = _load().orc_beam_search_batch(_p(X), X.shape[0], X.shape[1], _p(adj), adj.shape[1],
                                       metric, _p(Q), nq, _p(seeds), seeds.shape[1], ef, k,
                                       _p(ids), _p(dd), _p(ndc), _p(nexp), _p(mg), threads)
    _check(rc, "beam_search")
    return ids, dd, ndc, nexp, mg


def medoid(X, metric=L2) -> int:
    X = _f32(X)
    return int(_load().orc_medoid(_p(X), X.shape[0], X.shape[1], metric))


def prune(X, owners, W, R, alpha, metric=L2, keep_all_if_fit=False, threads=0):
    """Occlusion prune of each owner's pool.  Returns out [nv,R], margin [nv]."""
    X = _f32(X)
    owners = np.ascontiguousarray(owners, dtype=np.int64)
    W = _i32(np.atleast_2d(W))
    out = np.empty((owners.shape[0], R), np.int32)
    mg = np.empty(owners.shape[0], np.float64)
    rc = _load().orc_prune_batch(_p(X), X.shape[1], metric, _p(owners), owners.shape[0], _p(W),
                                 W.shape[1], R, alpha, int(keep_all_if_fit), _p(out), _p(mg),
                                 threads)
    _check(rc, "prune")
    return out, mg


def reverse_edges(X, lists, eu, ev, alpha, metric=L2, threads=0):
    """Adds reverse edges u <- v into a copy of lists [N,R]; returns it."""
    X = _f32(X)
    lists = np.array(lists, dtype=np.int32, copy=True, order="C")
    eu, ev = _i32(eu), _i32(ev)
    rc = _load().orc_reverse_edges(_p(X), X.shape[1], metric, _p(lists), lists.shape[1], _p(eu),
                                   _p(ev), eu.shape[0], alpha, threads)
    _check(rc, "reverse_edges")
    return lists


def expand(X, adj, k_plus, metric=L2, threads=0):
    """Neighbour expansion N+(v) [n,k_plus]; also ndc, expansions, margin."""
    X, adj = _f32(X), _i32(adj)
    n = X.shape[0]
    out = np.empty((n, k_plus), np.int32)
    ndc = np.empty(n, np.int64)
    nexp = np.empty(n, np.int64)
    mg = np.empty(n, np.float64)
    rc = _load().orc_expand(_p(X), n, X.shape[1], _p(adj), adj.shape[1], metric, k_plus, _p(out),
                            _p(ndc), _p(nexp), _p(mg), threads)
    _check(rc, "expand")
    return out, ndc, nexp, mg


def reverse_knn(nplus, k):
    """R_k CSR (offs [n+1] int64, ids) from the first k columns of N+."""
    nplus = _i32(nplus)
    n, kp = nplus.shape
    offs = np.empty(n + 1, np.int64)
    ids = np.empty(max(1, n * k), np.int32)
    _check(_load().orc_reverse_knn(_p(nplus), n, kp, k, _p(offs), _p(ids)), "reverse_knn")
    return offs, ids[: offs[-1]].copy()


def select_pivots(n, offs, ids):
    """Lazy greedy (Algorithm 2, Phase 2).  Returns pivot_of [n] (-1 = pivot),
    pivots in selection order, count of pivots with an earlier pivot in R_k."""
    offs = np.ascontiguousarray(offs, dtype=np.int64)
    ids = _i32(ids) if len(ids) else np.zeros(1, np.int32)
    piv_of = np.empty(n, np.int32)
    piv = np.empty(max(1, n), np.int32)
    npiv = np.zeros(1, np.int64)
    dep = np.zeros(1, np.int64)
    _check(_load().orc_select_pivots(n, _p(offs), _p(ids), _p(piv_of), _p(piv), _p(npiv),
                                     _p(dep)), "select_pivots")
    return piv_of, piv[: npiv[0]].copy(), int(dep[0])


def idps_cost(D, A, in_P, gamma, beta) -> float:
    D = np.ascontiguousarray(D, dtype=np.float64)
    A = np.ascontiguousarray(A, dtype=np.uint8)
    in_P = np.ascontiguousarray(in_P, dtype=np.uint8)
    return float(_load().orc_idps_cost(D.shape[0], _p(D), _p(A), _p(in_P), gamma, beta))


def build_graph(X, R, L, alpha, metric=L2, batch_max=None, threads=0):
    """Batch-synchronous two-stage PG build.  Returns (adj [n,R] int32, entry)."""
    X = _f32(X)
    n = X.shape[0]
    if batch_max is None:
        batch_max = default_batch_max(n)
    adj = np.empty((n, R), np.int32)
    ep = np.zeros(1, np.int32)
    rc = _load().orc_build(_p(X), n, X.shape[1], metric, R, L, alpha, batch_max, _p(adj), _p(ep),
                           threads)
    _check(rc, "build")
    return adj, int(ep[0])


def default_batch_max(n: int) -> int:
    """Round size cap of the batch-synchronous build: n/64 clamped to
    [64, 1024] (the library's default)."""
    return min(1024, max(64, n // 64))


def bruteforce_knn(X, Q, k, metric=L2, threads=0):
    X, Q = _f32(X), _f32(Q)
    ids = np.empty((Q.shape[0], k), np.int32)
    dd = np.empty((Q.shape[0], k), np.float64)
    rc = _load().orc_bruteforce_knn(_p(X), X.shape[0], X.shape[1], metric, _p(Q), Q.shape[0], k,
                                    _p(ids), _p(dd), threads)
    _check(rc, "bruteforce_knn")
    return ids, dd


def rnsm_merge(segments, graphs, entries, plan, R, L, alpha, metric=L2, k_rev=5, k_plus=None,
               ef_slide=None, c_cross=None, threads=0, cm=False, union_prune=False):
    """Algorithm 2 over the pairs of ``plan`` [(src, dst), ...] in order.

    segments: list of [n_s, d] float32; graphs: list of [n_s, r_in] int32
    (local ids); entries: local entry vertex per segment.  Returns the merged
    graph [N, R] in global ids (segment-concatenation order) and stats.
    cm=True runs the Cross-query Merge comparator (Section 3.1) instead:
    every source vertex runs a naive search of the target (no expansion,
    pivots or sliding), then the same prune and reverse edges.
    union_prune=True runs the multi-pair union variant: the searches of every
    plan edge, then one prune per source vertex over its list and the first
    c_cross results of each of its edges, then one reverse-edge pass."""
    p = default_params(R, L, k_rev, k_plus, ef_slide, c_cross)
    X = _f32(np.concatenate(segments, axis=0))
    sizes = np.array([s.shape[0] for s in segments], np.int64)
    seg_off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    r_in = graphs[0].shape[1]
    adj = _i32(np.concatenate([np.asarray(g, np.int32) for g in graphs], axis=0))
    ent = _i32(entries)
    ps = _i32([a for a, _ in plan]) if plan else np.zeros(1, np.int32)
    pd = _i32([b for _, b in plan]) if plan else np.zeros(1, np.int32)
    out = np.empty((X.shape[0], R), np.int32)
    st = np.zeros(8, np.int64)
    rc = _load().orc_rnsm_merge(_p(X), X.shape[1], _p(seg_off), len(segments), _p(adj), r_in,
                                _p(ent), metric, R, L, alpha, p["k_rev"], p["k_plus"],
                                p["ef_slide"], p["c_cross"], _p(ps), _p(pd), len(plan), _p(out),
                                _p(st), threads, int(bool(cm)), int(bool(union_prune)))
    _check(rc, "rnsm_merge")
    keys = ["ndc_expand", "ndc_search", "nexp_expand", "nexp_search", "pivots", "followers",
            "dependent_pivots", "reverse_edges"]
    return out, dict(zip(keys, (int(v) for v in st)))


def default_params(R, L, k_rev=5, k_plus=None, ef_slide=None, c_cross=None):
    """Parameter defaults: k_plus = max(2k, 16), ef_slide = ceil(L/2), c_cross = ef_slide."""
    k_plus = k_plus or max(2 * k_rev, 16)
    ef_slide = ef_slide or (L + 1) // 2
    c_cross = c_cross or ef_slide
    return {"R": R, "L": L, "k_rev": k_rev, "k_plus": k_plus, "ef_slide": ef_slide,
            "c_cross": c_cross}


def pair_plan(sizes):
    """Single-pair orientation: the smaller segment is the source (equal sizes:
    the larger index)."""
    a, b = 0, 1
    if sizes[0] < sizes[1]:
        return [(0, 1)]
    return [(1, 0)]


def mos(C, Rm, Delta):
    """Algorithm 3 on a cost matrix: edges in insertion order and their
    degree-bound violation flags."""
    C = np.ascontiguousarray(C, dtype=np.float64)
    m = C.shape[0]
    cap = m * m
    ea = np.empty(cap, np.int32)
    eb = np.empty(cap, np.int32)
    fl = np.empty(cap, np.int32)
    ne = np.zeros(1, np.int32)
    _check(_load().orc_mos(m, _p(C), Rm, Delta, _p(ea), _p(eb), _p(fl), _p(ne), cap), "mos")
    k = int(ne[0])
    return [(int(a), int(b)) for a, b in zip(ea[:k], eb[:k])], fl[:k].astype(bool)


def mos_plan(sizes, centroids=None, Rm=0, Delta=0):
    """Ordered, oriented merge plan [(src, dst, cost), ...]."""
    sizes = np.ascontiguousarray(sizes, dtype=np.int64)
    m = sizes.shape[0]
    cen = None if centroids is None else _f32(centroids)
    D = 0 if cen is None else cen.shape[1]
    cap = max(1, m * m)
    src = np.empty(cap, np.int32)
    dst = np.empty(cap, np.int32)
    cost = np.empty(cap, np.float64)
    n = np.zeros(1, np.int32)
    _check(_load().orc_mos_plan(m, _p(sizes), _p(cen), D, Rm, Delta, _p(src), _p(dst), _p(cost),
                                _p(n), cap), "mos_plan")
    k = int(n[0])
    return [(int(a), int(b), float(c)) for a, b, c in zip(src[:k], dst[:k], cost[:k])]


def recall_at_k(found_ids, found_pool, gt_dist, Q, k=10, metric=L2):
    """Tie-tolerant Recall@k (Eq. recall_at_k): a returned id counts if its
    FP64 distance to the query is within the true k-th NN distance.
    found_ids index ``found_pool`` (the vector table searched)."""
    found_pool, Q = _f32(found_pool), _f32(Q)
    hit = 0
    for qi in range(Q.shape[0]):
        dk = gt_dist[qi, k - 1]
        for r in found_ids[qi, :k]:
            if r >= 0 and distance(found_pool[r], Q[qi], metric) <= dk:
                hit += 1
    return hit / (k * Q.shape[0])
