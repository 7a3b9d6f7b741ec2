"""The C-ABI library on the host: it loads, exports every declared entry
point, its host planners (pivot selection, MOS) equal the oracle's, and host
validation rejects bad arguments before any device work.  CPU only."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import oracle
from workloads import generators as gen

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def rn():
    from paper_2602_17099_gb300 import build as b
    b.build()
    from paper_2602_17099_gb300 import rnsm
    rnsm.lib()
    return rnsm


def _declared():
    with open(os.path.join(ROOT, "include", "rnsm.h")) as f:
        src = f.read()
    return sorted(set(re.findall(r"RNSM_API\s+[\w\s\*]+?\b(\w+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for must in ["rnsm_merge", "mos_plan", "rnsm_workspace_size", "rnsm_build_segment",
                 "rnsm_search", "rnsm_last_error"]:
        assert must in names


def test_library_exports_every_declared_symbol(rn):
    lib = rn.lib()
    for name in _declared():
        assert hasattr(lib, name), name
    assert set(_declared()) <= set(rn.exported_symbols())
    assert "sm_103a" in rn.version()


@pytest.mark.parametrize("seed", range(3))
def test_host_pivot_selection_equals_oracle(rn, seed):
    X = gen.gaussian(800, 8, 200 + seed)
    adj, _ = oracle.build_graph(X, 10, 20, 1.2)
    nplus, _, _, _ = oracle.expand(X, adj, 12)
    for k in (1, 3, 5):
        offs, ids = oracle.reverse_knn(nplus, k)
        want_of, want_piv, _ = oracle.select_pivots(800, offs, ids)
        got_of, got_piv = rn.select_pivots(800, offs, ids)
        np.testing.assert_array_equal(got_of, want_of)
        np.testing.assert_array_equal(got_piv, want_piv)


@pytest.mark.parametrize("m", [1, 2, 3, 5, 8, 10, 17, 50])
def test_host_mos_plan_equals_oracle(rn, m):
    rng = np.random.default_rng(m)
    sizes = rng.integers(50, 5000, m)
    cen = rng.standard_normal((m, 6)).astype(np.float32)
    for c in (None, cen):
        want = oracle.mos_plan(sizes, c)
        got = rn.mos_plan(sizes, c)
        assert [(a, b) for a, b, _ in got] == [(a, b) for a, b, _ in want]
        np.testing.assert_allclose([x for _, _, x in got], [x for _, _, x in want], rtol=0,
                                   atol=0)


def test_host_mos_plan_equal_sizes_orientation(rn):
    assert [(a, b) for a, b, _ in rn.mos_plan([7, 7])] == [(1, 0)]
    assert [(a, b) for a, b, _ in rn.mos_plan([3, 9])] == [(0, 1)]


def test_host_validation_rejects_bad_arguments(rn):
    lib = rn.lib()
    p = rn.params(16, 32)
    seg = rn.Segment(10, 32, 16, 0, 0, 0)    # NULL vectors
    segs = (rn.Segment * 1)(seg)
    st = lib.rnsm_merge(segs, 1, C.byref(p), None, 0, None, None, None)
    assert st == rn.EINVAL and b"NULL" in lib.rnsm_last_error()
    bad = rn.params(0, 32)
    st = lib.rnsm_merge(segs, 1, C.byref(bad), None, 0, None, None, None)
    assert st == rn.EINVAL and b"R=0" in lib.rnsm_last_error()
    bad = rn.params(16, 32, c_cross=40, ef_slide=16)
    st = lib.rnsm_merge(segs, 1, C.byref(bad), None, 0, None, None, None)
    assert st == rn.EINVAL
    n = C.c_int32(0)
    st = lib.mos_plan(0, None, None, 0, 0, 0, None, C.byref(n))
    assert st == rn.EINVAL
    # capacity too small
    sizes = np.array([5, 6, 7, 8], np.int64)
    cap = C.c_int32(1)
    out = (rn.MosEdge * 1)()
    st = lib.mos_plan(4, sizes.ctypes.data_as(C.c_void_p), None, 0, 0, 0, out, C.byref(cap))
    assert st == rn.EINVAL and cap.value > 1
    offs = np.array([0, 1, 2], np.int64)
    ids = np.array([1, 5], np.int32)   # 5 is out of range
    po = np.empty(2, np.int32)
    pv = np.empty(2, np.int32)
    npv = C.c_int64(0)
    st = lib.rnsm_select_pivots(2, offs.ctypes.data_as(C.c_void_p), ids.ctypes.data_as(C.c_void_p),
                                po.ctypes.data_as(C.c_void_p), pv.ctypes.data_as(C.c_void_p),
                                C.byref(npv))
    assert st == rn.EGRAPH


def test_unsupported_dimension_is_rejected(rn):
    lib = rn.lib()
    p = rn.params(16, 32)
    seg = rn.Segment(10, 36, 16, 16, 16, 0)   # dim 36 has no kernel
    segs = (rn.Segment * 1)(seg)
    st = lib.rnsm_merge(segs, 1, C.byref(p), None, 0, C.c_void_p(16), None, None)
    assert st == rn.EINVAL and b"dim=36" in lib.rnsm_last_error()
