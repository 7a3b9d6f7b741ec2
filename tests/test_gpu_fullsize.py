"""The headline workload at full size (SIFT-like 2 x 500k, d = 128, R = 32,
L = 64, alpha = 1.2), in the launch configuration the benchmark times.

The oracle cannot merge a million rows in test time, so this file checks what
it can compute one by one, and properties that hold at any size:

* the merged graph: ids in range, no self loops, no duplicate ids per row,
  out-degree <= R, rows of the source segment in (distance, id) order and
  obeying the occlusion rule (no kept s before c with alpha d(s,c) <= d(v,c)),
  with exact FP64 distances on sampled rows (integer data: FP32 is exact);
* the beam search over the full target graph with 70,000 queries (the
  autotuned launch shape): sampled queries equal the oracle's Algorithm 1 bit
  for bit;
* the prune over 100,000 owners with pools of R + 32 candidates: sampled
  owners equal the oracle's prune;
* determinism: a second merge gives the same graph.
"""
import numpy as np
import pytest
import torch

import oracle
from workloads import generators as gen

pytestmark = pytest.mark.gpu

R, L, ALPHA = 32, 64, 1.2


@pytest.fixture(scope="module")
def rn():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_17099_gb300 import build as b
    b.build()
    from paper_2602_17099_gb300 import rnsm
    return rnsm


@pytest.fixture(scope="module")
def full(rn):
    segs, _ = gen.sift_case(n_per_seg=500_000, nq=10)
    vd = [torch.from_numpy(s).cuda() for s in segs]
    graphs = [rn.build_segment(v, R, L, ALPHA) for v in vd]
    tsegs = [(v, g, e) for v, (g, e) in zip(vd, graphs)]
    out, st = rn.merge(tsegs, rn.params(R, L, ALPHA))
    return segs, vd, graphs, tsegs, out, st


def test_full_size_merge_invariants_and_occlusion_rule(rn, full):
    segs, vd, graphs, tsegs, out, st = full
    N = sum(len(s) for s in segs)
    o = out.long()
    assert out.shape == (N, R)
    assert bool(((o >= -1) & (o < N)).all())
    rows = torch.arange(N, device=o.device)[:, None]
    assert not bool((o == rows).any())                       # no self loops
    s_, _ = torch.sort(o, dim=1)
    dup = (s_[:, 1:] == s_[:, :-1]) & (s_[:, 1:] >= 0)
    assert not bool(dup.any())                               # no duplicate ids
    assert st["reverse_edges"] > 0 and st["pivots"] > 0
    # the source is the segment with the larger index (equal sizes); its rows
    # come straight out of the occlusion prune
    X = np.concatenate(segs).astype(np.float64)
    lists = out.cpu().numpy()
    rng = np.random.default_rng(0)
    src0 = len(segs[0])
    for v in rng.choice(np.arange(src0, N), 400, replace=False):
        ids = lists[v][lists[v] >= 0]
        d = ((X[ids] - X[v]) ** 2).sum(1)
        key = np.lexsort((ids, d))
        assert (key == np.arange(len(ids))).all(), v          # (distance, id) order
        for j in range(1, len(ids)):
            dsc = ((X[ids[:j]] - X[ids[j]]) ** 2).sum(1)
            assert not (ALPHA * dsc <= d[j]).any(), (v, j)      # kept edges pass the rule


def test_full_size_search_parity_sampled(rn, full):
    segs, vd, graphs, tsegs, out, st = full
    T, (gT, eT) = vd[0], graphs[0]
    rng = np.random.default_rng(1)
    qi = rng.choice(len(segs[1]), 70_000, replace=False)
    Q = torch.from_numpy(segs[1][qi]).cuda()
    seeds = torch.full((len(qi), 1), eT, dtype=torch.int32, device="cuda")
    ids, dd, _ = rn.search(T, gT, Q, seeds, L, L)
    pick = rng.choice(len(qi), 120, replace=False)
    wid, wd, _, _, _ = oracle.beam_search(segs[0], gT.cpu().numpy(), segs[1][qi[pick]],
                                          np.full((len(pick), 1), eT, np.int32), L, L)
    np.testing.assert_array_equal(ids.cpu().numpy()[pick], wid)
    np.testing.assert_array_equal(dd.cpu().numpy()[pick].astype(np.float64), wd)


def test_full_size_prune_parity_sampled(rn, full):
    segs, vd, graphs, tsegs, out, st = full
    X = torch.cat(vd)
    n0 = len(segs[0])
    rng = np.random.default_rng(2)
    owners = rng.choice(len(segs[1]), 100_000, replace=False).astype(np.int32) + n0
    g1 = graphs[1][0].cpu().numpy()
    # pool: the owner's input list (global ids) and 32 random vertices of the other segment
    pool = np.concatenate([np.where(g1[owners - n0] >= 0, g1[owners - n0] + n0, -1),
                           rng.integers(0, n0, size=(len(owners), 32)).astype(np.int32)], axis=1)
    got = rn.prune(X, torch.from_numpy(owners).cuda(), torch.from_numpy(pool).cuda(), R, ALPHA)
    pick = rng.choice(len(owners), 300, replace=False)
    want, _ = oracle.prune(np.concatenate(segs), owners[pick].astype(np.int64), pool[pick], R, ALPHA)
    np.testing.assert_array_equal(got.cpu().numpy()[pick], want)


def test_full_size_merge_is_deterministic(rn, full):
    segs, vd, graphs, tsegs, out, st = full
    again, _ = rn.merge(tsegs, rn.params(R, L, ALPHA))
    assert torch.equal(again, out)
