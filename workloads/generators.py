"""Seeded synthetic inputs for the RNSM merge path.

This module is shared by the FP64 oracle's tests and by the CUDA path's tests
and benchmark.  It holds random-number recipes only: no distance, search,
prune or ordering arithmetic of the merge method lives here.

The paper measures on SIFT, DEEP, GIST, IMAGE, ANTON and MARCO (Section 6,
Table "Dataset Statistics").  None of those datasets is available, so every
workload below is a seeded stand-in with the same dimension, scale, value
distribution and partition type (random vs cluster partitions, Section 3.1).

Workloads (sizes are parameters so the same recipe serves small parity cases):

* ``gaussian``      -- iid N(0,1) rows (the tiny parity case, d=32).
* ``sift_like``     -- 1,000 low-rank Gaussian clusters rounded and clipped to
                       integers 0..255, d=128 (SIFT stand-in).  Every value is
                       an integer, so squared-L2 distances are exact in FP32.
* ``deep_like``     -- unit-norm d=96 mixture of low-rank clusters (DEEP stand-in).
* ``embed_like``    -- unit-norm d=768 mixture of anisotropic Gaussians
                       (IMAGE embedding stand-in, inner product).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "gaussian",
    "sift_like",
    "deep_like",
    "deep_like_gpu_segments",
    "embed_like",
    "random_partition",
    "cluster_partition",
    "lognormal_sizes",
    "tiny_case",
    "sift_case",
]


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def gaussian(n: int, d: int, seed: int) -> np.ndarray:
    """iid N(0,1) rows, float32, shape [n, d]."""
    return _rng(seed).standard_normal((n, d), dtype=np.float64).astype(np.float32)


def sift_like(n: int, seed: int, d: int = 128, n_comp: int = 1000, rank: int = 32,
              scale: float = 4.0, noise: float = 3.0) -> np.ndarray:
    """Integer-valued mixture of low-rank Gaussian clusters, values 0..255.

    x = clip(round(c_j + A_j z + noise * eps), 0, 255) with centers
    c_j ~ U[0,128]^d, A_j a d x rank matrix of N(0, scale^2) entries,
    z ~ N(0, I_rank), eps ~ N(0, I_d), uniform component weights.  The low
    rank puts the local intrinsic dimensionality near 18 (SIFT: 19.4 in the
    paper's dataset table); isotropic clusters in 128 dimensions sit near 40
    and their proximity graphs lose navigability at SIFT scale."""
    g = _rng(seed)
    centers = g.uniform(0.0, 128.0, size=(n_comp, d))
    A = g.standard_normal((n_comp, d, rank)) * scale
    comp = g.integers(0, n_comp, size=n)
    z = g.standard_normal((n, rank))
    eps = g.standard_normal((n, d), dtype=np.float32)
    out = np.empty((n, d), dtype=np.float32)
    order = np.argsort(comp, kind="stable")
    bounds = np.searchsorted(comp[order], np.arange(n_comp + 1))
    for j in range(n_comp):
        rows = order[bounds[j]:bounds[j + 1]]
        if rows.size:
            out[rows] = (centers[j] + z[rows] @ A[j].T).astype(np.float32)
    out += np.float32(noise) * eps
    np.clip(np.rint(out, out=out), 0.0, 255.0, out=out)
    return out


def _normalise(x: np.ndarray) -> np.ndarray:
    nrm = np.sqrt(np.einsum("ij,ij->i", x, x))
    nrm[nrm == 0.0] = 1.0
    return x / nrm[:, None]


def deep_like(n: int, seed: int, d: int = 96, n_comp: int = 1000, rank: int = 32,
              scale: float = 0.06, noise: float = 0.01, return_components: bool = False,
              chunk: int = 1 << 18):
    """Unit-norm mixture of low-rank Gaussian clusters (DEEP stand-in).

    x = normalise(mu_j + A_j z + noise * eps): means mu_j ~ N(0, I) normalised,
    A_j a d x rank matrix of N(0, scale^2) entries, z ~ N(0, I_rank),
    eps ~ N(0, I_d), uniform component weights.  The defaults put the local
    intrinsic dimensionality near 19.5 (DEEP in the paper's dataset table);
    isotropic clusters of the same spread sit near 50 in 96 dimensions.

    With ``return_components`` the component index of each row and the
    component means are returned too (used by the cluster partition)."""
    g = _rng(seed)
    means = _normalise(g.standard_normal((n_comp, d)))
    A = g.standard_normal((n_comp, d, rank)) * scale
    comp_all = g.integers(0, n_comp, size=n)
    out = np.empty((n, d), dtype=np.float32)
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        comp = comp_all[s:e]
        z = g.standard_normal((e - s, rank))
        x = means[comp] + noise * g.standard_normal((e - s, d))
        order = np.argsort(comp, kind="stable")
        bounds = np.searchsorted(comp[order], np.arange(n_comp + 1))
        for j in range(n_comp):
            rows = order[bounds[j]:bounds[j + 1]]
            if rows.size:
                x[rows] += z[rows] @ A[j].T
        out[s:e] = _normalise(x).astype(np.float32)
    if return_components:
        return out, comp_all, means
    return out


def deep_like_gpu_segments(n: int, nq: int, seed: int, sizes, part_seed: int, device="cuda",
                           d: int = 96, n_comp: int = 1000, rank: int = 32, scale: float = 0.06,
                           noise: float = 0.01, chunk: int = 1 << 15, stream: bool = False,
                           return_all: bool = False):
    """The DEEP stand-in's recipe (deep_like) drawn with a seeded torch
    generator on `device`, for workloads of tens of GB: the same mixture and
    parameters, other random numbers.  Rows 0..n-1 are cluster-partitioned as
    in cluster_partition (components sorted by a random projection of their
    means, assigned contiguously to segments of the given sizes) and written in
    partition order into one tensor; the segments are views of it (rows in
    ascending order within a segment).  With ``stream`` the rows stay in the
    order they are drawn (arrival order) and segment k is the next sizes[k]
    rows.  Returns (segments, queries), plus the whole tensor with
    ``return_all``."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    f32 = dict(device=device, dtype=torch.float32)

    def normalise(x):
        return x / x.norm(dim=1, keepdim=True).clamp_min(1e-30)

    means = normalise(torch.randn(n_comp, d, generator=g, **f32))
    A = torch.randn(n_comp, d, rank, generator=g, **f32) * scale
    comp = torch.randint(0, n_comp, (n + nq,), generator=g, device=device)
    gp = torch.Generator(device=device)
    gp.manual_seed(part_seed)
    proj = means @ torch.randn(d, generator=gp, **f32)
    comp_rank = torch.empty(n_comp, dtype=torch.int64, device=device)
    comp_rank[torch.argsort(proj, stable=True)] = torch.arange(n_comp, device=device)
    order = torch.argsort(comp_rank[comp[:n]], stable=True)   # ties by row id
    sizes_t = torch.as_tensor(np.asarray(sizes, dtype=np.int64), device=device)
    bounds = torch.cat([torch.zeros(1, dtype=torch.int64, device=device), torch.cumsum(sizes_t, 0)])
    # destination of every row: its segment's start + its rank among that segment's rows
    if stream:
        dest = torch.arange(n, dtype=torch.int64, device=device)
    else:
        dest = torch.empty(n, dtype=torch.int64, device=device)
        for k in range(len(sizes)):
            rows = torch.sort(order[bounds[k]:bounds[k + 1]]).values
            dest[rows] = bounds[k] + torch.arange(rows.numel(), device=device)
    del order
    allx = torch.empty((n, d), **f32)
    Q = torch.empty((nq, d), **f32)
    for s in range(0, n + nq, chunk):
        e = min(n + nq, s + chunk)
        c = comp[s:e]
        z = torch.randn(e - s, rank, generator=g, **f32)
        x = means[c] + noise * torch.randn(e - s, d, generator=g, **f32)
        x += torch.bmm(A[c], z.unsqueeze(2)).squeeze(2)
        x = normalise(x)
        e0 = min(e, n)
        if s < e0:
            allx[dest[s:e0]] = x[:e0 - s]
        if e > n:
            lo = max(s, n)
            Q[lo - n:e - n] = x[lo - s:]
    segs = [allx[int(bounds[k]):int(bounds[k + 1])] for k in range(len(sizes))]
    if return_all:
        return segs, Q, allx
    return segs, Q


def embed_like(n: int, seed: int, d: int = 768, n_comp: int = 2000,
               rank: int = 32, noise: float = 0.013) -> np.ndarray:
    """Unit-norm anisotropic mixture: x = normalise(mu_j + A_j z + noise*eps),
    A_j a d x rank matrix with singular values 0.3 * 0.9^i, z ~ N(0, I_rank).
    The noise level puts the local intrinsic dimensionality near 21 (IMAGE in
    the paper's dataset table: 21.2)."""
    g = _rng(seed)
    means = _normalise(g.standard_normal((n_comp, d)))
    sv = 0.3 * (0.9 ** np.arange(rank))
    comp = g.integers(0, n_comp, size=n)
    z = g.standard_normal((n, rank)) * sv[None, :]
    out = np.empty((n, d), dtype=np.float32)
    order = np.argsort(comp, kind="stable")
    bounds = np.searchsorted(comp[order], np.arange(n_comp + 1))
    for j in range(n_comp):
        rows = order[bounds[j]:bounds[j + 1]]
        if not rows.size:
            continue
        # orthonormal column basis of component j (QR of a Gaussian matrix)
        basis, _ = np.linalg.qr(g.standard_normal((d, rank)))
        x = means[j] + z[rows] @ basis.T + noise * g.standard_normal((rows.size, d))
        out[rows] = _normalise(x).astype(np.float32)
    return out


def random_partition(n: int, m: int, seed: int) -> list[np.ndarray]:
    """Equal-size random split of row indices 0..n-1 into m parts (Section 3.1)."""
    perm = _rng(seed).permutation(n)
    return [np.sort(p) for p in np.array_split(perm, m)]


def lognormal_sizes(m: int, total: int, lo: int, hi: int, seed: int,
                    sigma: float = 0.6) -> np.ndarray:
    """m segment sizes ~ lognormal(sigma), rescaled to ``total``, clipped to [lo, hi]."""
    g = _rng(seed)
    w = g.lognormal(0.0, sigma, size=m)
    sizes = np.clip(np.rint(w / w.sum() * total), lo, hi).astype(np.int64)
    # Spread the rounding / clipping remainder evenly over the segments that can
    # still move in its direction (lowest indices take the odd rows), until the
    # sizes sum to `total` or every segment sits at its bound.
    diff = int(total - sizes.sum())
    while diff != 0:
        free = [j for j in range(m) if (sizes[j] < hi if diff > 0 else sizes[j] > lo)]
        if not free:
            break
        q, r = divmod(abs(diff), len(free))
        for idx, j in enumerate(free):
            want = q + (1 if idx < r else 0)
            room = (hi - sizes[j]) if diff > 0 else (sizes[j] - lo)
            step = min(want, int(room))
            sizes[j] += step if diff > 0 else -step
        diff = int(total - sizes.sum())
    return sizes


def cluster_partition(comp: np.ndarray, means: np.ndarray, sizes: np.ndarray,
                      seed: int) -> list[np.ndarray]:
    """Cluster partition: components sorted by a random projection of their
    means, their rows assigned contiguously to fill each segment in turn."""
    g = _rng(seed)
    proj = means @ g.standard_normal(means.shape[1])
    comp_rank = np.empty(len(means), dtype=np.int64)
    comp_rank[np.argsort(proj, kind="stable")] = np.arange(len(means))
    order = np.lexsort((np.arange(len(comp)), comp_rank[comp]))
    bounds = np.concatenate([[0], np.cumsum(sizes)])
    return [np.sort(order[bounds[i]:bounds[i + 1]]) for i in range(len(sizes))]


def tiny_case(n_per_seg: int = 5000, d: int = 32, seed_data: int = 1, seed_query: int = 2,
              nq: int = 1000):
    """2 x n_per_seg iid N(0,1) rows; segment 0 = first half, segment 1 = second half."""
    X = gaussian(2 * n_per_seg, d, seed_data)
    Q = gaussian(nq, d, seed_query)
    return [X[:n_per_seg].copy(), X[n_per_seg:].copy()], Q


def sift_case(n_per_seg: int = 500_000, m: int = 2, seed_data: int = 3, seed_query: int = 4,
              nq: int = 10_000, d: int = 128):
    """SIFT-like integer mixture, random partition into m equal segments.

    The queries come from the same mixture (same centers and sigmas)."""
    n = n_per_seg * m
    X = sift_like(n + nq, seed_data, d=d)
    Q = X[n:].copy()
    X = X[:n]
    parts = random_partition(n, m, seed_data + 1000)
    del seed_query  # queries share the mixture draw above
    return [X[p].copy() for p in parts], Q
