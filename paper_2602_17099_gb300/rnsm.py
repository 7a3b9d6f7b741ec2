"""Python binding of librnsm (include/rnsm.h): argument marshalling only.

Every function takes torch CUDA tensors (or host objects where the C ABI
takes host memory), passes raw pointers and the current CUDA stream to the C
ABI, and raises :class:`RnsmError` on a non-OK status.  There is no CPU
path: if the compiled library is missing, loading raises immediately.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(os.environ.get("RNSM_BUILD_DIR") or os.path.join(_HERE, "_build"),
                        "librnsm.so")

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, EGRAPH = range(6)
L2, IP = 0, 1
FP32, BF16, FP8 = 0, 1, 2
FLAG_CM = 0x1
FLAG_HOST_PIVOTS = 0x2
FLAG_GRAPH = 0x4
FLAG_UNION = 0x8
_STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ETIMEOUT", 5: "EGRAPH"}


class RnsmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"RNSM_{_STATUS.get(status, status)}: {msg}")
        self.status = status


class Segment(C.Structure):
    _fields_ = [("n", C.c_int64), ("dim", C.c_int32), ("r_in", C.c_int32),
                ("vecs", C.c_void_p), ("adj", C.c_void_p), ("entry", C.c_int32)]


class Params(C.Structure):
    _fields_ = [("R", C.c_int32), ("L", C.c_int32), ("alpha", C.c_float),
                ("metric", C.c_int32), ("prec", C.c_int32), ("k_rev", C.c_int32),
                ("k_plus", C.c_int32), ("ef_slide", C.c_int32), ("c_cross", C.c_int32),
                ("flags", C.c_uint32)]


class MosEdge(C.Structure):
    _fields_ = [("src", C.c_int32), ("dst", C.c_int32), ("cost", C.c_double)]


class Stats(C.Structure):
    _fields_ = [("wall_s", C.c_double), ("host_pivot_s", C.c_double), ("ndc", C.c_int64),
                ("expansions", C.c_int64), ("rechecks", C.c_int64), ("pivots", C.c_int64),
                ("followers", C.c_int64), ("reverse_edges", C.c_int64),
                ("launches", C.c_int64), ("phase_ms", C.c_double * 8),
                ("search_ndc", C.c_int64 * 3), ("search_exp", C.c_int64 * 3),
                ("search_queries", C.c_int64 * 3), ("tile_error", C.c_double * 4),
                ("tile_tests", C.c_int64), ("prune_kernel", C.c_int32 * 2)]

    def as_dict(self):
        out = {}
        for k, _ in self._fields_:
            v = getattr(self, k)
            out[k] = list(v) if hasattr(v, "__len__") else v
        return out


_lib = None
_lock = threading.Lock()

P = C.c_void_p
i32, i64, f32 = C.c_int32, C.c_int64, C.c_float
_SIGS = {
    "mos_plan": (i32, [i32, P, P, i32, i32, i32, P, P]),
    "rnsm_merge": (i32, [P, i32, P, P, i32, P, P, P]),
    "rnsm_workspace_size": (C.c_size_t, [P, i32, P]),
    "rnsm_release_workspace": (None, []),
    "rnsm_search": (i32, [P, i64, i32, P, i32, P, i64, P, i32, i32, i32, i32, P, P, P, P]),
    "rnsm_expand": (i32, [P, i64, i32, P, i32, i32, i32, P, P]),
    "rnsm_reverse_knn": (i32, [P, i64, i32, i32, P, P, P]),
    "rnsm_select_pivots": (i32, [i64, P, P, P, P, P]),
    "rnsm_select_pivots_gpu": (i32, [P, i64, i32, i32, P, P, P, P, P, P]),
    "rnsm_prune": (i32, [P, i64, i32, P, i64, P, i32, i32, f32, i32, i32, i32, P, P]),
    "rnsm_reverse_edges": (i32, [P, i64, i32, P, i32, P, P, i64, f32, i32, P]),
    "rnsm_prune_noalloc": (i32, [P, i64, i32, P, i64, P, i32, i32, f32, i32, i32, P, P]),
    "rnsm_build_segment": (i32, [P, i64, i32, P, i64, P, P, P]),
    "rnsm_medoid": (i32, [P, i64, i32, i32, P, P]),
    "rnsm_last_error": (C.c_char_p, []),
    "rnsm_version": (C.c_char_p, []),
}


def lib():
    """The loaded librnsm (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    f"librnsm.so not found at {LIB_PATH}: build it first "
                    "(python -m paper_2602_17099_gb300.build); there is no CPU fallback")
            h = C.CDLL(LIB_PATH)
            for name, (res, args) in _SIGS.items():
                fn = getattr(h, name)
                fn.restype = res
                fn.argtypes = args
            _lib = h
    return _lib


def exported_symbols():
    return list(_SIGS)


def _check(status):
    if status != OK:
        raise RnsmError(status, lib().rnsm_last_error().decode())


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dev(t: torch.Tensor, dtype, name):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return C.c_void_p(t.data_ptr())


def _ptr_or_none(t, dtype, name):
    return None if t is None else _dev(t, dtype, name)


def params(R, L, alpha=1.2, metric=L2, prec=FP32, k_rev=0, k_plus=0, ef_slide=0, c_cross=0,
           flags=0) -> Params:
    return Params(R, L, alpha, metric, prec, k_rev, k_plus, ef_slide, c_cross, flags)


def segment(vecs: torch.Tensor, adj: torch.Tensor, entry: int) -> Segment:
    _dev(vecs, torch.float32, "vecs")
    _dev(adj, torch.int32, "adj")
    return Segment(vecs.shape[0], vecs.shape[1], adj.shape[1], vecs.data_ptr(), adj.data_ptr(),
                   int(entry))


def mos_plan(sizes, centroids=None, degree_bound=0, diameter_bound=0):
    sizes = np.ascontiguousarray(sizes, dtype=np.int64)
    m = sizes.shape[0]
    cen = None if centroids is None else np.ascontiguousarray(centroids, dtype=np.float32)
    cap = max(1, m * m)
    out = (MosEdge * cap)()
    n = C.c_int32(cap)
    _check(lib().mos_plan(m, sizes.ctypes.data_as(P), None if cen is None else cen.ctypes.data_as(P),
                          0 if cen is None else cen.shape[1], degree_bound, diameter_bound, out,
                          C.byref(n)))
    return [(out[i].src, out[i].dst, out[i].cost) for i in range(n.value)]


def merge(segments, p: Params, plan=None, out: torch.Tensor | None = None):
    """RNSM over ``plan`` [(src, dst), ...] (None: the 2-segment default).

    segments: list of (vecs [n,d] f32 cuda, adj [n,r_in] i32 cuda, entry).
    Returns (merged adjacency [N, R] int32 on the device, stats dict)."""
    segs = (Segment * len(segments))(*[segment(v, a, e) for v, a, e in segments])
    N = sum(int(v.shape[0]) for v, _, _ in segments)
    dev = segments[0][0].device
    if out is None:
        out = torch.empty((N, p.R), dtype=torch.int32, device=dev)
    _dev(out, torch.int32, "out")
    if plan is None:
        cplan, nplan = None, 0
    else:
        cplan = (MosEdge * max(1, len(plan)))(*[MosEdge(int(e[0]), int(e[1]),
                                                        float(e[2]) if len(e) > 2 else 0.0)
                                                for e in plan])
        nplan = len(plan)
    st = Stats()
    _check(lib().rnsm_merge(segs, len(segments), C.byref(p), cplan, nplan,
                            C.c_void_p(out.data_ptr()), _stream(), C.byref(st)))
    return out, st.as_dict()


def workspace_size(segments, p: Params) -> int:
    segs = (Segment * len(segments))(*[segment(v, a, e) for v, a, e in segments])
    return int(lib().rnsm_workspace_size(segs, len(segments), C.byref(p)))


def release_workspace():
    lib().rnsm_release_workspace()


def search(vecs, adj, queries, seeds, ef, k, metric=L2, want_dists=True, want_ndc=False):
    """Batched beam search; seeds [nq, n_seeds] int32 (-1 = none)."""
    nq = queries.shape[0]
    if seeds.dim() == 1:
        seeds = seeds.view(-1, 1)
    ids = torch.empty((nq, k), dtype=torch.int32, device=vecs.device)
    dd = torch.empty((nq, k), dtype=torch.float32, device=vecs.device) if want_dists else None
    ndc = torch.empty(nq, dtype=torch.int64, device=vecs.device) if want_ndc else None
    _check(lib().rnsm_search(_dev(vecs, torch.float32, "vecs"), vecs.shape[0], vecs.shape[1],
                             _dev(adj, torch.int32, "adj"), adj.shape[1],
                             _dev(queries, torch.float32, "queries"), nq,
                             _dev(seeds, torch.int32, "seeds"), seeds.shape[1], ef, k, metric,
                             C.c_void_p(ids.data_ptr()), _ptr_or_none(dd, torch.float32, "d"),
                             _ptr_or_none(ndc, torch.int64, "ndc"), _stream()))
    return ids, dd, ndc


def expand(vecs, adj, k_plus, metric=L2):
    out = torch.empty((vecs.shape[0], k_plus), dtype=torch.int32, device=vecs.device)
    _check(lib().rnsm_expand(_dev(vecs, torch.float32, "vecs"), vecs.shape[0], vecs.shape[1],
                             _dev(adj, torch.int32, "adj"), adj.shape[1], k_plus, metric,
                             C.c_void_p(out.data_ptr()), _stream()))
    return out


def reverse_knn(nplus, k):
    n, kp = nplus.shape
    offs = torch.empty(n + 1, dtype=torch.int64, device=nplus.device)
    ids = torch.empty(max(1, n * k), dtype=torch.int32, device=nplus.device)
    _check(lib().rnsm_reverse_knn(_dev(nplus, torch.int32, "nplus"), n, kp, k,
                                  C.c_void_p(offs.data_ptr()), C.c_void_p(ids.data_ptr()),
                                  _stream()))
    return offs, ids[: int(offs[-1].item())]


def select_pivots(n, offs, ids):
    """Host lazy greedy on numpy CSR; returns (pivot_of, pivots)."""
    offs = np.ascontiguousarray(offs, dtype=np.int64)
    ids = np.ascontiguousarray(ids, dtype=np.int32)
    if ids.size == 0:
        ids = np.zeros(1, np.int32)
    piv_of = np.empty(n, np.int32)
    piv = np.empty(max(1, n), np.int32)
    npiv = C.c_int64(0)
    _check(lib().rnsm_select_pivots(n, offs.ctypes.data_as(P), ids.ctypes.data_as(P),
                                    piv_of.ctypes.data_as(P), piv.ctypes.data_as(P),
                                    C.byref(npiv)))
    return piv_of, piv[: npiv.value].copy()


def select_pivots_gpu(nplus, k, offs, ids):
    """Device pivot selection on device N+ and R_k CSR; returns
    (pivot_of tensor, number of pivots, rounds)."""
    n, kp = nplus.shape
    piv_of = torch.empty(n, dtype=torch.int32, device=nplus.device)
    npiv = C.c_int64(0)
    rounds = C.c_int32(0)
    _check(lib().rnsm_select_pivots_gpu(_dev(nplus, torch.int32, "nplus"), n, kp, k,
                                        _dev(offs, torch.int64, "offs"),
                                        _dev(ids, torch.int32, "ids"),
                                        C.c_void_p(piv_of.data_ptr()), C.byref(npiv),
                                        C.byref(rounds), _stream()))
    return piv_of, npiv.value, rounds.value


def prune(vecs, owners, pool, R, alpha, metric=L2, keep_all_if_fit=False, prec=FP32):
    nv = owners.shape[0]
    out = torch.empty((nv, R), dtype=torch.int32, device=vecs.device)
    _check(lib().rnsm_prune(_dev(vecs, torch.float32, "vecs"), vecs.shape[0], vecs.shape[1],
                            _dev(owners, torch.int32, "owners"), nv,
                            _dev(pool, torch.int32, "pool"), pool.shape[1], R, alpha, metric,
                            int(keep_all_if_fit), prec, C.c_void_p(out.data_ptr()), _stream()))
    return out


NOALLOC_MAX_OWNERS = 262144


def prune_noalloc(vecs, owners, pool, R, alpha, metric=L2, keep_all_if_fit=False, out=None):
    """rnsm_prune without device allocation inside the library (the caller
    provides ``out``; scratch is the library's static device array)."""
    nv = owners.shape[0]
    if out is None:
        out = torch.empty((nv, R), dtype=torch.int32, device=vecs.device)
    elif tuple(out.shape) != (nv, R) or out.device != vecs.device:
        # the kernel writes nv * R ids: a smaller or foreign buffer would be
        # written past its end or on the wrong device
        raise ValueError(f"out must have shape ({nv}, {R}) on {vecs.device}, "
                         f"got {tuple(out.shape)} on {out.device}")
    _check(lib().rnsm_prune_noalloc(_dev(vecs, torch.float32, "vecs"), vecs.shape[0],
                                    vecs.shape[1], _dev(owners, torch.int32, "owners"), nv,
                                    _dev(pool, torch.int32, "pool"), pool.shape[1], R, alpha,
                                    metric, int(keep_all_if_fit), _dev(out, torch.int32, "out"),
                                    _stream()))
    return out


def reverse_edges(vecs, lists, eu, ev, alpha, metric=L2):
    """Adds reverse edges u <- v into ``lists`` in place."""
    _check(lib().rnsm_reverse_edges(_dev(vecs, torch.float32, "vecs"), vecs.shape[0],
                                    vecs.shape[1], _dev(lists, torch.int32, "lists"),
                                    lists.shape[1], _dev(eu, torch.int32, "eu"),
                                    _dev(ev, torch.int32, "ev"), eu.shape[0], alpha, metric,
                                    _stream()))
    return lists


def build_segment(vecs, R, L, alpha=1.2, metric=L2, batch_max=0):
    """Batch-synchronous two-stage PG build; returns (adj [n,R] int32 cuda, entry)."""
    out = torch.empty((vecs.shape[0], R), dtype=torch.int32, device=vecs.device)
    ent = C.c_int32(0)
    p = params(R, L, alpha, metric)
    _check(lib().rnsm_build_segment(_dev(vecs, torch.float32, "vecs"), vecs.shape[0],
                                    vecs.shape[1], C.byref(p), batch_max,
                                    C.c_void_p(out.data_ptr()), C.byref(ent), _stream()))
    return out, ent.value


def medoid(vecs, metric=L2) -> int:
    ent = C.c_int32(0)
    _check(lib().rnsm_medoid(_dev(vecs, torch.float32, "vecs"), vecs.shape[0], vecs.shape[1],
                             metric, C.byref(ent), _stream()))
    return ent.value


def version() -> str:
    return lib().rnsm_version().decode()
