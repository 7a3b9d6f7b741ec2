"""The FP32 walk-over-kept-rows prune (pools of at most 64 raw candidates,
d <= 128), forced through RNSM_PRUNE_VARIANT=3: bit-exact against the oracle
on integer rows, and identical to the triangle kernel (variant 0) on real
rows, inner product, every dimension class, duplicates, -1 and the owner in
the pool, R = 1 and R = 64, pools that overflow to the general kernel, the
reverse-edge pools and a whole merge."""
import numpy as np
import pytest
import torch

import oracle
from workloads import generators as gen

pytestmark = pytest.mark.gpu


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


def _pools(n, w, seed, nown):
    rng = np.random.default_rng(seed)
    owners = rng.choice(n, nown, replace=False).astype(np.int32)
    pool = rng.integers(-1, n, size=(nown, w)).astype(np.int32)
    if w > 5:
        pool[:, 3] = owners          # the owner itself is dropped
        pool[:, 5] = pool[:, 4]      # a duplicate is dropped
    return owners, pool


def _both(rn, monkeypatch, *args, **kw):
    monkeypatch.setenv("RNSM_PRUNE_VARIANT", "3")
    walk = host(rn.prune(*args, **kw))
    monkeypatch.setenv("RNSM_PRUNE_VARIANT", "0")
    tri = host(rn.prune(*args, **kw))
    monkeypatch.delenv("RNSM_PRUNE_VARIANT", raising=False)
    return walk, tri


@pytest.mark.parametrize("R,w,alpha", [(32, 64, 1.2), (16, 40, 1.0), (1, 64, 1.2),
                                       (64, 64, 1.5), (5, 7, 2.0), (32, 200, 1.2)])
def test_walk_exact_on_integer_data(rn, monkeypatch, R, w, alpha):
    X = gen.sift_like(3000, 5, d=128)
    owners, pool = _pools(3000, w, R + w, 301)
    want, _ = oracle.prune(X, owners.astype(np.int64), pool, R, alpha)
    walk, tri = _both(rn, monkeypatch, dev(X), dev(owners), dev(pool), R, alpha)
    np.testing.assert_array_equal(walk, want)
    np.testing.assert_array_equal(tri, want)
    want2, _ = oracle.prune(X, owners.astype(np.int64), pool, R, alpha, keep_all_if_fit=True)
    walk2, _ = _both(rn, monkeypatch, dev(X), dev(owners), dev(pool), R, alpha,
                     keep_all_if_fit=True)
    np.testing.assert_array_equal(walk2, want2)


@pytest.mark.parametrize("d,metric", [(4, 0), (32, 0), (96, 0), (100, 0), (128, 0),
                                      (96, 1), (128, 1), (36, 1)])
def test_walk_equals_triangle_on_real_rows(rn, monkeypatch, d, metric):
    X = gen.deep_like(4000, d, d=d) if metric == 1 else gen.gaussian(4000, d, d)
    owners, pool = _pools(4000, 64, 7 * d + metric, 3000)
    for R, alpha in ((32, 1.2), (8, 1.0), (64, 1.3)):
        walk, tri = _both(rn, monkeypatch, dev(X), dev(owners), dev(pool), R, alpha, metric=metric)
        np.testing.assert_array_equal(walk, tri, err_msg=f"R {R} alpha {alpha}")


def test_walk_degenerate_pools(rn, monkeypatch):
    # all -1; all the owner; all one id; a single candidate; identical rows
    X = gen.sift_like(500, 9, d=64)
    X[100:140] = X[100]
    owners = np.arange(6, dtype=np.int32)
    pool = np.full((6, 64), -1, np.int32)
    pool[1, :] = 1
    pool[2, :] = 77
    pool[3, 0] = 9
    pool[4, :40] = np.arange(100, 140)
    pool[5, :] = np.arange(200, 264)
    want, _ = oracle.prune(X, owners.astype(np.int64), pool, 16, 1.2)
    walk, tri = _both(rn, monkeypatch, dev(X), dev(owners), dev(pool), 16, 1.2)
    np.testing.assert_array_equal(walk, want)
    np.testing.assert_array_equal(tri, want)


def test_walk_on_reverse_edge_pools_and_merge(rn, monkeypatch):
    # the reverse-edge prune (pools of the list plus incoming edges, some over
    # 64 and sent on to the general kernel), then a whole 2-segment merge
    X = gen.sift_like(6000, 3, d=128)
    adj, _ = oracle.build_graph(X, 32, 64, 1.2)
    rng = np.random.default_rng(4)
    eu = rng.integers(0, 6000, 40000).astype(np.int32)
    ev = rng.integers(0, 6000, 40000).astype(np.int32)
    eu[:3000] = 17
    keep = eu != ev
    pairs = np.unique(np.stack([eu[keep], ev[keep]], 1), axis=0)
    eu, ev = pairs[:, 0].copy(), pairs[:, 1].copy()
    want = oracle.reverse_edges(X, adj.copy(), eu, ev, 1.2)
    monkeypatch.setenv("RNSM_PRUNE_VARIANT", "3")
    got = dev(adj.copy())
    rn.reverse_edges(dev(X), got, dev(eu), dev(ev), 1.2)
    np.testing.assert_array_equal(host(got), want)

    segs = []
    for k in range(2):
        v = dev(X[3000 * k:3000 * (k + 1)])
        a, e = rn.build_segment(v, 32, 64, 1.2)
        segs.append((v, a, e))
    g3, _ = rn.merge(segs, rn.params(32, 64, 1.2))
    monkeypatch.setenv("RNSM_PRUNE_VARIANT", "0")
    g0, _ = rn.merge(segs, rn.params(32, 64, 1.2))
    monkeypatch.delenv("RNSM_PRUNE_VARIANT", raising=False)
    np.testing.assert_array_equal(host(g3), host(g0))
