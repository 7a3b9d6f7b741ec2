"""The error bounds of the tensor-core prune tiles, checked by emulation on
the CPU (the BF16 pair tile at L2; the general tile's inner-product rows).

The pair tile decides an occlusion test from the tile only when the tile's
distance d~(s, c) = G_ss + G_cc - 2 G_sc is within kappa (n_s + n_c)^2 of the
FP32 prune distance d_fp32(s, c) (the two-chain definition).  This test
emulates what the tile computes -- rows centred on the owner in FP32, split
into hi = bf16(y) and lo = bf16(y - hi), the Gram of hi + lo accumulated with
one FP32 rounding per 16-wide MMA step -- and the FP32 chains, on real-valued
and integer-valued pools, and checks that the bound (with the constants of the
derivation: staging residual kE, accumulation e1, FP32 chain gam) covers every
pair.  It checks the derivation, not the kernel; the kernel is checked by the
GPU parity tests (identical graphs in BF16 and FP32 mode)."""
import numpy as np
import pytest

from workloads import generators as gen


def bf16_rn(x):
    """Round float32 values to bfloat16 (nearest, ties to even), as float32."""
    b = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    rounded = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return rounded.astype(np.uint32).view(np.float32)


def fma32(a, b, c):
    # a*b is exact in float64; one rounding of a*b + c to float64, then float32
    # (the double rounding can differ from a true fma in rare ties; the bound's
    # margin covers that)
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(np.float32)


def fp32_prune_dist(a, b):
    """Two chains over v - x: E over even dimensions, O over odd, then E + O."""
    y = (a[:, None, :] - b[None, :, :]).astype(np.float32)
    e = np.zeros(y.shape[:2], np.float32)
    o = np.zeros(y.shape[:2], np.float32)
    for k in range(0, y.shape[2], 2):
        e = fma32(y[..., k], y[..., k], e)
        o = fma32(y[..., k + 1], y[..., k + 1], o)
    return (e + o).astype(np.float32)


def tile(rows, owner):
    """Centred rows split in hi / lo and their Gram, one FP32 rounding per
    16-wide step of the accumulation."""
    y = (owner[None, :] - rows).astype(np.float32)
    hi = bf16_rn(y)
    lo = bf16_rn((y - hi).astype(np.float32))
    four = bool(np.any(lo != 0))
    x = (hi.astype(np.float64) + lo.astype(np.float64))
    d = rows.shape[1]
    G = np.zeros((len(rows), len(rows)), np.float32)
    for k0 in range(0, d, 16):
        part = x[:, k0:k0 + 16] @ x[:, k0:k0 + 16].T          # exact products, summed in FP64
        G = (G.astype(np.float64) + part).astype(np.float32)
    return G, four


def bound_terms(dim, four):
    n_instr = (4 if four else 1) * (dim // 16)
    eps_c = 1.01 * (n_instr + 1) * 2.0 ** -22
    e1 = 1.01 * eps_c
    kE = 1.0002 * (2.0 ** -16 + 2.0 ** -24) if four else 1.0001 * 2.0 ** -24
    gam = 1.01 * (dim + 2) * 2.0 ** -24
    kappa = 1.01 * (e1 + 2 * kE + kE * kE + gam * (1 + kE) ** 2)
    return e1, kappa


@pytest.mark.parametrize("kind,d", [("deep", 96), ("deep", 128), ("gauss", 64), ("sift", 128),
                                    ("embed", 128)])
def test_tile_distance_within_its_bound(kind, d):
    n = 65 * 24
    X = {"deep": lambda: gen.deep_like(n, 11, d=d),
         "gauss": lambda: gen.gaussian(n, d, 12),
         "sift": lambda: gen.sift_like(n, 13, d=d),
         "embed": lambda: gen.embed_like(n, 14, d=d, n_comp=20)}[kind]().astype(np.float32)
    worst = 0.0
    for g in range(0, n, 65):
        owner, rows = X[g], X[g + 1:g + 65]
        G, four = tile(rows, owner)
        e1, kappa = bound_terms(d, four)
        diag = np.diag(G).astype(np.float64)
        dt = diag[:, None] + diag[None, :] - 2.0 * G.astype(np.float64)
        n2 = np.maximum(diag, 0.0) * (1 + 2 * e1)
        nr = np.sqrt(n2)
        B = kappa * (nr[:, None] + nr[None, :]) ** 2
        d32 = fp32_prune_dist(rows, rows).astype(np.float64)
        err = np.abs(dt - d32)
        off = ~np.eye(len(rows), dtype=bool)
        assert (err[off] <= B[off]).all(), (kind, d, g)
        worst = max(worst, float((err[off] / B[off]).max()))
        # the owner distance the kernel computes exactly equals the tile's diagonal
        # within the same bound (n_c alone)
        dv = fp32_prune_dist(owner[None, :], rows)[0].astype(np.float64)
        assert (np.abs(diag - dv) <= kappa * n2 + 1e-30).all(), (kind, d, g)
    assert worst < 1.0


def test_integer_rows_spanning_256_need_no_lo_term():
    # the hi-only instantiation's premise: integer components spanning at most
    # 256 give differences that bf16 holds exactly
    X = gen.sift_like(2000, 15, d=128).astype(np.float32) + np.float32(1000.0)
    assert X.max() - X.min() <= 256
    y = (X[:1000] - X[1000:]).astype(np.float32)
    assert np.array_equal(bf16_rn(y), y)
    # one step past the range is no longer exact
    assert bf16_rn(np.float32(257.0)) != np.float32(257.0)


def ip_chain(a, b):
    """The FP32 prune distance for inner product: two chains of fma(a_k, b_k),
    then 1 - (E + O)."""
    e = np.zeros((len(a), len(b)), np.float32)
    o = np.zeros((len(a), len(b)), np.float32)
    for k in range(0, a.shape[1], 2):
        e = fma32(a[:, None, k], b[None, :, k], e)
        o = fma32(a[:, None, k + 1], b[None, :, k + 1], o)
    return (np.float32(1.0) - (e + o)).astype(np.float32)


@pytest.mark.parametrize("d,terms", [(768, 2), (256, 1)])
def test_general_tile_inner_product_bound(d, terms):
    # the general tile's inner-product rows: stored hi (and lo) terms, residual
    # norm E = ||x - hi - lo|| (rounded up), row norm ||x||; the Gram of the
    # staged terms in FP32 steps of 16 products; bound of the kernel:
    #   1.01 (n_s E_c + E_s n_c + E_s E_c + eps_c (n_s + E_s)(n_c + E_c) + gam n_s n_c + 2^-23)
    X = gen.embed_like(64 * 4, 16, d=d, n_comp=8).astype(np.float32)
    hi = bf16_rn(X)
    lo = bf16_rn((X - hi).astype(np.float32)) if terms == 2 else np.zeros_like(X)
    res = (X.astype(np.float64) - hi - lo)
    E = np.sqrt((res ** 2).sum(1)) * 1.001 + 1e-30
    nrm = np.sqrt((X.astype(np.float64) ** 2).sum(1)) * 1.0001
    x = hi.astype(np.float64) + lo.astype(np.float64)
    n_instr = (4 if terms == 2 else 1) * (d // 16)
    eps_c = 1.01 * (n_instr + 1) * 2.0 ** -22
    gam = 1.01 * (d + 2) * 2.0 ** -24
    worst = 0.0
    for g in range(0, len(X), 64):
        idx = slice(g, g + 64)
        G = np.zeros((64, 64), np.float32)
        for k0 in range(0, d, 16):
            G = (G.astype(np.float64) + x[idx, k0:k0 + 16] @ x[idx, k0:k0 + 16].T).astype(np.float32)
        dt = 1.0 - G.astype(np.float64)
        d32 = ip_chain(X[idx], X[idx]).astype(np.float64)
        ns, es = nrm[idx], E[idx]
        B = 1.01 * (ns[:, None] * es[None, :] + es[:, None] * ns[None, :] + es[:, None] * es[None, :]
                    + eps_c * (ns[:, None] + es[:, None]) * (ns[None, :] + es[None, :])
                    + gam * ns[:, None] * ns[None, :] + 1.2e-7)
        err = np.abs(dt - d32)
        assert (err <= B).all(), (d, terms, g)
        worst = max(worst, float((err / B).max()))
    assert worst < 1.0
