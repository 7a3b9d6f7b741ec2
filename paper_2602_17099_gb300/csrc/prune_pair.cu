// K4b: the BF16 / FP8 tensor-core prune for small pools (L2, at most 64 raw
// candidates, dimension a multiple of 16 (BF16) or 32 (FP8) up to 128), two
// owners per tile.
//
// The general tensor-core prune (prune_tc.cu) gives one CTA of eight warps to
// one owner and spends most of its time in barrier-separated phases; for pools
// of 64 candidates at d <= 128 the FP32 small-pool kernel was faster.  This
// kernel packs two owners into one 128 x 128 Gram tile and keeps every phase
// inside the two warps that own the candidates' TMEM lanes:
//
//  1. Pool.  Slot t of owner o gets its id; a repeated id keeps its first slot
//     (match_any in a warp, a 32-entry scan across the two warps), so the
//     remaining (distance, id) keys are distinct.
//  2. One pass per row, in slot order.  The slot's thread reads its FP32 row
//     once: v - x feeds the two chains of the FP32 prune distance (the
//     definition of common.cuh), giving the exact owner distance, and the same
//     v - x (the row centred on the owner, rounded once) is split into
//     hi = bf16(y) and lo = bf16(y - hi) and written into the K-major
//     no-swizzle tile: rows 0..63 are owner A's slots, rows 64..127 owner B's.
//     If every lo of the pair is zero only hi.hi is multiplied; when the whole
//     table is integer-valued with a range of at most 256 the kernel is
//     instantiated without lo terms at all (kHiOnly).
//  3. One thread issues the MMAs (hi.hi, plus lo.hi, hi.lo and lo.lo) of the
//     tile against itself, M = N = 128, into 128 TMEM columns, and commits
//     them to an mbarrier (the wait is bounded by 1 s).  Meanwhile every slot
//     builds the mask of the slots before it in (distance, id) order: the
//     order is exact, so no owner-distance interval logic is needed.
//  4. Warp w reads TMEM lanes 32w..32w+31, i.e. 32 slots s of one owner, and
//     that owner's 64 columns c.  From the centred Gram G:
//     d~(s, c) = G_ss + G_cc - 2 G_sc, with |d~ - d_fp32(s, c)| <=
//     kappa (n_s + n_c)^2 <= b_s + b_c, n_r^2 a bound on the squared norm of
//     the staged row r (from G_rr).  A test "s occludes c" (s before c) is
//     settled by the tile when alpha (d~ +- (b_s + b_c)) - d(v, c) has one
//     sign, else by a tighter per-pair bound, else by the exact FP32
//     distance with the FP32 prune's own rule fmaf(alpha, d, -d(v, c)) <= 0.
//     The ballots of a column are the occluder bits of c by slot.
//  5. One warp per owner runs the greedy walk in ballot rounds on slot masks
//     (as the FP32 small-pool kernel does on positions); a kept slot's output
//     index is the number of kept slots before it, and the cap keeps the
//     first R.  The other warp prefetches the next owner's rows into L2.
//
// FP8 (E4M3) tiles stage the same centred row in two E4M3 terms with a
// per-row power-of-two scale sigma_r (the largest with sigma_r max|y| <= 448,
// found in a first pass over the row that also runs the FP32 chain):
// hi = e4m3(sigma_r y), lo = e4m3(sigma_r y - hi); the MMAs (kind::f8f6f4,
// K = 32) accumulate sigma_s sigma_c (hi + lo)_s . (hi + lo)_c, and the tile
// values are unscaled by 1 / (sigma_s sigma_c), exactly (powers of two).  Two
// E4M3 terms carry 8 significant bits: integer differences of magnitude <= 256
// are staged exactly (the same whole-table check as the BF16 hi-only case),
// otherwise the staging error is at most about 2^-8 of the row.
//
// The result equals the FP32 prune's: the order is exact, and every
// occlusion decision either follows from a proven bound or is taken in FP32.
//
// Bound (per pair s, c; x~ the staged row, x the centred FP32 row):
//   staging   |x~ - (x_c - x_v)| <= kE |x~| element-wise, kE = 1.0002 (2^-16 + 2^-24)
//             (2^-24 (1.0001) when every lo is zero);
//             FP8: ||x~ - (x_c - x_v)|| <= kE ||x~||, kE = 1.01 (1.004 2^-8 + 2^-24 + c),
//             c = sqrt(dim) 2^-10 / 224 covering E4M3 subnormals (half their
//             spacing, 2^-10, against a scaled row of max |.| >= 224), or the
//             hi-only constant when the whole table is integer with range <= 256;
//   Gram      |G~_ij - x~_i . x~_j| <= e1 n_i n_j, e1 = 1.01 eps_c, eps_c =
//             1.01 (n_instr + 1) 2^-22 (the per-MMA-instruction accumulation
//             model of the general kernel; sampled tile statistics check it);
//   FP32      |d_fp32 - d| <= gam d, gam = 1.01 (dim + 2) 2^-24;
//   so |d~ - d_fp32| <= kappa (n_s + n_c)^2, kappa = 1.01 (e1 + 2 kE + kE^2 + gam (1 + kE)^2).
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <float.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "internal.h"
#include "tcgen05.cuh"

namespace rnsm {

namespace {

constexpr int kQT = 128;           // threads; warp w reads TMEM lanes 32w..32w+31
constexpr int kQC = 64;            // raw pool entries per owner
constexpr int kQCols = 128;        // TMEM columns (N = 128)
constexpr int kQMaxDim = 128;
constexpr uint64_t kQWaitNs = 1000000000ull;   // an MMA group takes microseconds
constexpr int kQErrEvery = 256;    // owners between two tile-error samples (FP64 is slow here)
constexpr int kQOpen = 64;         // open tests a warp queues per owner before deciding inline

struct PairSmem {
    alignas(16) float vrow[2][kQMaxDim];   // the owners' FP32 rows
    unsigned long long key[2][kQC];        // (distance bits, id) of each slot; ~0: none
    unsigned long long ltm[2][kQC];        // slots before each slot in (distance, id) order
    const float *rp[2][kQC];               // FP32 row of each slot
    float sd[2][kQC];                      // exact owner distance of each slot
    float gd[2][kQC];                      // Gram diagonal
    float nn[2][kQC];                      // bound on the staged row's squared norm
    float2 pq[2][kQC];                     // column terms of the occlusion test
    float isc[2][kQC];                     // FP8: 1 / sigma of each slot's staged row
    uint32_t occ[2][kQC][2];               // occluders of slot c, by slot
    uint2 open_q[4][kQOpen];               // per warp: tests the loose bound left open
                                           // (tile value, c | slot << 8)
    uint32_t live[2][2];                   // valid slots (ids not repeated), per warp
    uint64_t bar;
    uint32_t tmem_slot;
};

__device__ __forceinline__ void owner_sync(int o) {
    asm volatile("bar.sync %0, 64;" ::"r"(1 + o) : "memory");
}

__device__ __forceinline__ void max_pos(unsigned int *p, float v) {
    if (v > 0.f) atomicMax(p, __float_as_uint(v));
}

// The FP32 prune distance in FP64 (tile statistics only).
__device__ double dist64(const float *a, const float *b, int dim) {
    double acc = 0.0;
    for (int k = 0; k < dim; ++k) {
        const double d = (double)a[k] - (double)b[k];
        acc = fma(d, d, acc);
    }
    return acc;
}

// An occlusion test the loose bound left open: the tighter per-pair bound,
// then the exact FP32 decision.  Returns bit 0 = occluded, bit 1 = decided in FP32.
__device__ __noinline__ int decide_open(float g, float gs, float ns2, float gc, float nc2, float dvc,
                                        const float *rs, const float *rc, int dim, float alpha,
                                        float e1, float kE, float gam) {
    const float dsc = gs + gc - 2.0f * g;
    const float sn = sqrtf(ns2) + sqrtf(nc2);
    const float bc = e1 * sn * sn;                       // Gram accumulation
    const float E = kE * sn;                             // staging residual of both rows
    const float bq = E * (2.0f * sqrtf(fmaxf(dsc + bc, 0.f)) + E);
    const float bf = gam * (fmaxf(dsc, 0.f) + bc + bq);  // the FP32 chain's own rounding
    const float B = 1.01f * (bc + bq + bf) + 1e-6f * (gs + gc) + 1e-30f;
    const float slack = 1e-6f * (alpha * (fabsf(dsc) + B) + dvc);
    if (alpha * (dsc + B) - dvc + slack < 0.f) return 1;
    if (alpha * (dsc - B) - dvc - slack > 0.f) return 0;
    const float d = prune_dist(rs, rc, dim, 0);
    return (fmaf(alpha, d, -dvc) <= 0.f ? 1 : 0) | 2;
}

// Packs two floats into two E4M3 bytes (x in the low byte), rounding to
// nearest, saturating at 448.
__device__ __forceinline__ uint32_t e4m3x2(float x, float y) {
    return (uint32_t)__nv_cvt_float2_to_fp8x2(make_float2(x, y), __NV_SATFINITE, __NV_E4M3);
}
__device__ __forceinline__ float2 e4m3x2_to_float2(uint32_t v) {
    const __half2_raw h = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)v, __NV_E4M3);
    return __half22float2(*reinterpret_cast<const __half2 *>(&h));
}

// Largest power of two sigma with sigma * m <= 448 (1 for m = 0).
// (448 = 0.875 2^9; the exponent is capped so that sigma stays a normal float.)
__device__ __forceinline__ float e4m3_scale(float m) {
    if (!(m > 0.f)) return 1.f;
    int E;
    const float f = frexpf(m, &E);   // m = f 2^E, f in [0.5, 1)
    return ldexpf(1.0f, min((f <= 0.875f ? 9 : 8) - E, 126));
}

// kKind 0: BF16 hi and lo terms; 1: BF16 hi only -- every component of every
// row is an integer and their range is at most 256 (checked on the device
// before the launch), so y = x_c - x_v is exact in FP32 and in BF16 (half the
// shared memory); 2: two E4M3 terms with per-row power-of-two scales.
template <int kKind>
__global__ void __launch_bounds__(kQT, 4) prune_pair_kernel(const PruneArgs a, int chunk) {
    constexpr bool kHiOnly = kKind == 1;
    constexpr bool kF8 = kKind == 2;
    extern __shared__ __align__(1024) unsigned char tile[];
    __shared__ PairSmem s;
    __shared__ int64_t sh_i;
    __shared__ int sh_fail;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int o = warp >> 1, h = warp & 1, t = tid & 63;   // owner of the warp, half, thread in owner
    const int dim = a.dim, R = a.R;
    const float alpha = a.alpha;
    const int U = dim >> 3;                  // 16-byte units of a BF16 row
    const uint32_t esz = kF8 ? 1u : 2u;      // bytes per staged element
    const uint32_t SBO = 8u * esz * (uint32_t)dim;   // bytes between 8-row core-matrix bands
    const uint32_t region = 128u * esz * (uint32_t)dim;   // one term (hi or lo) of the tile
    const float gam = 1.01f * (float)(dim + 2) * 5.9604645e-08f;
    // FP8: the staging bound (the whole-table exact case reuses the hi-only constant)
    const float kE8 = a.pair_hi_only
                          ? 1.0001f * 5.9604645e-08f
                          : 1.01f * (1.004f * 3.90625e-03f + 5.9604645e-08f +
                                     sqrtf((float)dim) * 9.765625e-04f / 224.0f);

    if (tid == 0) {
        tc::mbar_init(&s.bar, 1);
        sh_fail = 0;
    }
    if (warp == 0) {
        tc::tmem_alloc(&s.tmem_slot, kQCols);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = s.tmem_slot;
    const uint32_t tbase = tc::smem_u32(tile);
    uint32_t phase = 0;
    unsigned long long rechecks = 0, tests = 0;

    for (;;) {
        if (tid == 0) sh_i = atomicAdd(a.work, chunk);
        __syncthreads();
        const int64_t i0 = sh_i;
        if (i0 >= a.n_owners || sh_fail) break;
        const int64_t i1 = min(a.n_owners, i0 + chunk);
        // the next owner of the chunk with a pool to prune (uniform over the CTA);
        // owners whose pools exceed the tile go to the overflow list
        int64_t cur = i0;
        auto next_owner = [&]() -> int64_t {
            while (cur < i1) {
                const int64_t j = cur++;
                int64_t cl = 0, ch = 0;
                if (a.csr_offs) {
                    cl = a.csr_offs[j];
                    ch = a.csr_offs[j + 1];
                }
                if (a.skip_empty_csr && ch == cl) continue;
                if ((int64_t)a.lenA + a.lenB + (ch - cl) > kQC) {
                    if (tid == 0) a.ovf_list[atomicAdd(a.ovf_count, 1ull)] = (int32_t)j;
                    continue;
                }
                return j;
            }
            return -1;
        };
        for (;;) {
            const int64_t j0 = next_owner();
            if (j0 < 0) break;
            const int64_t j1 = next_owner();
            const int64_t io = o == 0 ? j0 : j1;   // this warp pair's owner, -1: none
            // ---- 1. pool and owner row ------------------------------------------
            int32_t owner = -1;
            int nr = -1;
            int64_t c_lo = 0;
            if (io >= 0) {
                owner = a.owner_ids ? a.owner_ids[io] : (int32_t)(a.owner_base + io);
                int64_t c_hi = 0;
                if (a.csr_offs) {
                    c_lo = a.csr_offs[io];
                    c_hi = a.csr_offs[io + 1];
                }
                nr = (int)((int64_t)a.lenA + a.lenB + (c_hi - c_lo));
            }
            const float *orow = owner >= 0 ? seg_row(a.segs, owner, dim) : nullptr;
            const bool whole = nr >= 0 && a.keep_all_if_fit && nr <= R;   // no tests needed
            int32_t id = -1;
            if (t < nr) {
                if (t < a.lenA) {
                    id = a.listA[(int64_t)owner * a.lenA + t];
                } else if (t < a.lenA + a.lenB) {
                    id = a.listB[io * a.strideB + (t - a.lenA)];
                    if (id >= 0) id += a.offB;
                } else {
                    id = a.csr_ids[c_lo + (t - a.lenA - a.lenB)];
                }
                if (id == owner) id = -1;
            }
            if (orow)
                for (int k = t; k < dim; k += 64) s.vrow[o][k] = orow[k];
            s.occ[o][t][0] = 0u;
            s.occ[o][t][1] = 0u;
            // a repeated id keeps its first slot (same row, same distance: the FP32
            // prune keeps the first of equal (distance, id) entries)
            {
                const unsigned same = __match_any_sync(0xffffffffu, id);
                if (same & lanemask_lt()) id = -1;
                if (h == 0) s.key[o][t] = (unsigned long long)(uint32_t)id;   // ids only, for now
            }
            owner_sync(o);
            if (h == 1 && id >= 0) {
                for (int k = 0; k < 32; ++k)
                    if ((int32_t)(uint32_t)s.key[o][k] == id) id = -1;
            }
            const bool valid_t = id >= 0;
            // ---- 2. one pass over the row: exact owner distance and the tile terms
            const float *xrow = valid_t ? seg_row(a.segs, id, dim) : orow;
            const int r = 64 * o + t;   // tile row: this slot
            unsigned char *hrow = tile + (uint32_t)(r >> 3) * SBO + (uint32_t)(r & 7) * 16u;
            bool lo_any = false;
            float dxt = INFINITY;
            float isc_t = 1.f;
            if (!valid_t) {
                for (int u = 0; u < (kF8 ? U / 2 : U); ++u) {
                    *reinterpret_cast<uint4 *>(hrow + u * 128) = make_uint4(0u, 0u, 0u, 0u);
                    if (!kHiOnly)
                        *reinterpret_cast<uint4 *>(hrow + region + u * 128) = make_uint4(0u, 0u, 0u, 0u);
                }
            } else if (kF8 && a.pair_hi_only) {
                // integer rows spanning <= 256: |v - x| <= 256 is staged exactly with
                // sigma = 1, so one pass gives the FP32 prune distance (chains E and O
                // over v - x, in order) and the two terms
                f2_t acc = 0ull;
                const float *v = s.vrow[o];
                for (int u = 0; u < U / 2; ++u) {   // 16 dimensions per 16-byte unit
                    float4 x4[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) x4[q] = ldg4(xrow + 16 * u + 4 * q);
                    uint32_t hw[4], lw[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const float4 v4 = *reinterpret_cast<const float4 *>(v + 16 * u + 4 * q);
                        const f2_t y01 = f2_sub(f2_of(v4.x, v4.y), f2_of(x4[q].x, x4[q].y));
                        acc = f2_fma(y01, y01, acc);
                        const f2_t y23 = f2_sub(f2_of(v4.z, v4.w), f2_of(x4[q].z, x4[q].w));
                        acc = f2_fma(y23, y23, acc);
                        float z0, z1, z2, z3;
                        f2_split(y01, z0, z1);
                        f2_split(y23, z2, z3);
                        const uint32_t h01 = e4m3x2(z0, z1), h23 = e4m3x2(z2, z3);
                        const float2 f01 = e4m3x2_to_float2(h01), f23 = e4m3x2_to_float2(h23);
                        hw[q] = h01 | (h23 << 16);
                        lw[q] = e4m3x2(z0 - f01.x, z1 - f01.y) | (e4m3x2(z2 - f23.x, z3 - f23.y) << 16);
                    }
                    if (whole) {
                        hw[0] = hw[1] = hw[2] = hw[3] = 0u;
                        lw[0] = lw[1] = lw[2] = lw[3] = 0u;
                    }
                    lo_any |= ((lw[0] | lw[1] | lw[2] | lw[3]) & 0x7f7f7f7fu) != 0u;
                    *reinterpret_cast<uint4 *>(hrow + u * 128) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
                    *reinterpret_cast<uint4 *>(hrow + region + u * 128) =
                        make_uint4(lw[0], lw[1], lw[2], lw[3]);
                }
                dxt = chain2_final(acc, 0);
            } else if (kF8) {
                // pass 1: the FP32 prune distance (chains E and O over v - x, in order)
                // and max |v - x|; pass 2: the same v - x, scaled by sigma, in two terms
                f2_t acc = 0ull;
                float ymax = 0.f;
                const float *v = s.vrow[o];
                for (int u0 = 0; u0 < U; u0 += 4) {
                    float4 xa[4][2];
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        if (u0 + k < U) {
                            xa[k][0] = ldg4(xrow + 8 * (u0 + k));
                            xa[k][1] = ldg4(xrow + 8 * (u0 + k) + 4);
                        }
                    }
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const int u = u0 + k;
                        if (u >= U) break;
                        const float4 v0 = *reinterpret_cast<const float4 *>(v + 8 * u);
                        const float4 v1 = *reinterpret_cast<const float4 *>(v + 8 * u + 4);
                        const f2_t xs[4] = {f2_of(xa[k][0].x, xa[k][0].y), f2_of(xa[k][0].z, xa[k][0].w),
                                            f2_of(xa[k][1].x, xa[k][1].y), f2_of(xa[k][1].z, xa[k][1].w)};
                        const f2_t vs[4] = {f2_of(v0.x, v0.y), f2_of(v0.z, v0.w), f2_of(v1.x, v1.y),
                                            f2_of(v1.z, v1.w)};
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const f2_t y = f2_sub(vs[e], xs[e]);
                            acc = f2_fma(y, y, acc);
                            float y0, y1;
                            f2_split(y, y0, y1);
                            ymax = fmaxf(ymax, fmaxf(fabsf(y0), fabsf(y1)));
                        }
                    }
                }
                dxt = chain2_final(acc, 0);
                const float sg = e4m3_scale(ymax);
                isc_t = 1.0f / sg;   // a power of two: exact
                for (int u = 0; u < U / 2; ++u) {   // 16 dimensions per 16-byte unit
                    uint32_t hw[4], lw[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const float4 x4 = ldg4(xrow + 16 * u + 4 * q);
                        const float4 v4 = *reinterpret_cast<const float4 *>(v + 16 * u + 4 * q);
                        // y exactly as in pass 1, scaled exactly (sg is a power of two)
                        const float z0 = (v4.x - x4.x) * sg, z1 = (v4.y - x4.y) * sg;
                        const float z2 = (v4.z - x4.z) * sg, z3 = (v4.w - x4.w) * sg;
                        const uint32_t h01 = e4m3x2(z0, z1), h23 = e4m3x2(z2, z3);
                        const float2 f01 = e4m3x2_to_float2(h01), f23 = e4m3x2_to_float2(h23);
                        // z - hi is exact in FP32
                        const uint32_t l01 = e4m3x2(z0 - f01.x, z1 - f01.y);
                        const uint32_t l23 = e4m3x2(z2 - f23.x, z3 - f23.y);
                        hw[q] = h01 | (h23 << 16);
                        lw[q] = l01 | (l23 << 16);
                    }
                    if (whole) {   // no tests: the tile rows stay zero
                        hw[0] = hw[1] = hw[2] = hw[3] = 0u;
                        lw[0] = lw[1] = lw[2] = lw[3] = 0u;
                    }
                    lo_any |= ((lw[0] | lw[1] | lw[2] | lw[3]) & 0x7f7f7f7fu) != 0u;
                    *reinterpret_cast<uint4 *>(hrow + u * 128) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
                    *reinterpret_cast<uint4 *>(hrow + region + u * 128) =
                        make_uint4(lw[0], lw[1], lw[2], lw[3]);
                }
            } else {
                // the FP32 prune distance, chains E (even dimensions) and O (odd) over
                // v - x in increasing order, exactly as prune_dist; the same v - x,
                // split into hi + lo, is the staged row (centred on the owner)
                f2_t acc = 0ull;
                const float *v = s.vrow[o];
                // kRowBatch 16-byte units of the row in flight at a time
                constexpr int kRowBatch = 4;
                for (int u0 = 0; u0 < U; u0 += kRowBatch) {
                    float4 xa[kRowBatch][2];
#pragma unroll
                    for (int k = 0; k < kRowBatch; ++k) {
                        if (u0 + k < U) {
                            xa[k][0] = ldg4(xrow + 8 * (u0 + k));
                            xa[k][1] = ldg4(xrow + 8 * (u0 + k) + 4);
                        }
                    }
#pragma unroll
                    for (int k = 0; k < kRowBatch; ++k) {
                        const int u = u0 + k;
                        if (u >= U) break;
                        const float4 v0 = *reinterpret_cast<const float4 *>(v + 8 * u);
                        const float4 v1 = *reinterpret_cast<const float4 *>(v + 8 * u + 4);
                        const f2_t xs[4] = {f2_of(xa[k][0].x, xa[k][0].y), f2_of(xa[k][0].z, xa[k][0].w),
                                            f2_of(xa[k][1].x, xa[k][1].y), f2_of(xa[k][1].z, xa[k][1].w)};
                        const f2_t vs[4] = {f2_of(v0.x, v0.y), f2_of(v0.z, v0.w), f2_of(v1.x, v1.y),
                                            f2_of(v1.z, v1.w)};
                        uint32_t hw[4], lw[4];
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const f2_t y = f2_sub(vs[e], xs[e]);
                            acc = f2_fma(y, y, acc);
                            float y0, y1;
                            f2_split(y, y0, y1);
                            const __nv_bfloat162 hb = __floats2bfloat162_rn(y0, y1);
                            hw[e] = *reinterpret_cast<const uint32_t *>(&hb);
                            lw[e] = 0u;
                            if (!kHiOnly) {
                                const float2 hf = __bfloat1622float2(hb);
                                // y - hi is exact in FP32
                                float t0, t1;
                                f2_split(f2_sub(y, f2_of(hf.x, hf.y)), t0, t1);
                                const __nv_bfloat162 lb = __floats2bfloat162_rn(t0, t1);
                                lw[e] = *reinterpret_cast<const uint32_t *>(&lb);
                            }
                        }
                        if (whole) {   // no tests: the tile rows stay zero
                            hw[0] = hw[1] = hw[2] = hw[3] = 0u;
                            lw[0] = lw[1] = lw[2] = lw[3] = 0u;
                        }
                        *reinterpret_cast<uint4 *>(hrow + u * 128) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
                        if (!kHiOnly) {
                            lo_any |= ((lw[0] | lw[1] | lw[2] | lw[3]) & 0x7fff7fffu) != 0u;
                            *reinterpret_cast<uint4 *>(hrow + region + u * 128) =
                                make_uint4(lw[0], lw[1], lw[2], lw[3]);
                        }
                    }
                }
                dxt = chain2_final(acc, 0);
            }
            // distances are >= +0 (sums of squares), so their bit patterns order as the
            // values and (bits << 32 | id) orders as (distance, id); after the repeats are
            // dropped the valid keys are distinct
            const unsigned long long keyt =
                valid_t ? ((unsigned long long)__float_as_uint(dxt) << 32) | (uint32_t)id : ~0ull;
            {
                const unsigned lm = __ballot_sync(0xffffffffu, valid_t);
                if (lane == 0) s.live[o][h] = lm;
            }
            tc::fence_async_shared();
            tc::fence_before_sync();
            const bool four = __syncthreads_or(lo_any) != 0;   // ids read above are no longer needed
            tc::fence_after_sync();
            s.key[o][t] = keyt;
            s.sd[o][t] = dxt;
            s.rp[o][t] = xrow;
            if (kF8) s.isc[o][t] = isc_t;
            // ---- 3. the Gram tile -----------------------------------------------
            const int n_instr = (four ? 4 : 1) * (dim >> (kF8 ? 5 : 4));
            const float eps_c = 1.01f * (float)(n_instr + 1) * 2.384185791e-07f;
            const float e1 = 1.01f * eps_c;
            const float kE = kF8 ? kE8
                                 : four ? 1.0002f * (1.52587890625e-05f + 5.9604645e-08f)
                                        : 1.0001f * 5.9604645e-08f;
            const float kappa = 1.01f * (e1 + 2.0f * kE + kE * kE + gam * (1.0f + kE) * (1.0f + kE));
            const float cb = 2.0f * kappa + 1e-6f;
            if (tid == 0) {
                // one K-step = 32 bytes of each row: 16 BF16 or 32 E4M3 elements
                const uint32_t idesc = tc::instr_desc(kF8 ? 0u : 1u, 128, 128);
                for (int k = 0; k < (dim >> (kF8 ? 5 : 4)); ++k) {
                    const uint64_t dh = tc::smem_desc(tbase + k * 256, 128, SBO);
                    const uint64_t dl = tc::smem_desc(tbase + region + k * 256, 128, SBO);
                    if (kF8) {
                        tc::mma_fp8(taddr, dh, dh, idesc, k > 0 ? 1u : 0u);
                        if (four) {
                            tc::mma_fp8(taddr, dl, dh, idesc, 1u);
                            tc::mma_fp8(taddr, dh, dl, idesc, 1u);
                            tc::mma_fp8(taddr, dl, dl, idesc, 1u);
                        }
                    } else {
                        tc::mma_bf16(taddr, dh, dh, idesc, k > 0 ? 1u : 0u);
                        if (four) {
                            tc::mma_bf16(taddr, dl, dh, idesc, 1u);
                            tc::mma_bf16(taddr, dh, dl, idesc, 1u);
                            tc::mma_bf16(taddr, dl, dl, idesc, 1u);
                        }
                    }
                }
                if (!a.test_withhold_commit) tc::mma_commit(&s.bar);
            }
            // while the MMAs run: the slots before this one in (distance, id) order
            owner_sync(o);
            uint64_t ltm = 0ull;
            if (valid_t) {
#pragma unroll
                for (int k = 0; k < kQC; ++k) ltm |= s.key[o][k] < keyt ? 1ull << k : 0ull;
            }
            s.ltm[o][t] = ltm;
            {
                // one thread waits; the barrier passes the completion on to the others
                bool ok = true;
                if (tid == 0) ok = tc::mbar_wait_bounded(&s.bar, phase, kQWaitNs);
                if (__syncthreads_or(!ok)) {
                    if (tid == 0) {
                        atomicOr(a.err, 64);
                        sh_fail = 1;
                        // a second bounded chance for the MMAs before the tensor memory is freed
                        tc::mbar_wait_bounded(&s.bar, phase, kQWaitNs);
                    }
                    break;
                }
                phase ^= 1u;
            }
            tc::fence_after_sync();
            // ---- 4. occlusion tests from the tile ---------------------------------
            const uint32_t tl = taddr + ((uint32_t)(32 * warp) << 16);
            const int p = t;                         // this lane's slot (row s)
            float gs, ns2;
            {
                uint32_t ra[16], rb[16];
                tc::tmem_ld16(tl + 64 * o + 32 * h, ra);
                tc::tmem_ld16(tl + 64 * o + 32 * h + 16, rb);
                tc::tmem_wait_ld();
                float g = 0.f;
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    g = lane == q ? __uint_as_float(ra[q]) : g;
                    g = lane == q + 16 ? __uint_as_float(rb[q]) : g;
                }
                if (kF8) g *= isc_t * isc_t;   // exact: powers of two
                gs = g;
                ns2 = fmaxf(g, 0.f) * (1.0f + 2.0f * e1);
            }
            const float dvs = dxt;
            const float bs = cb * ns2;
            const float As = alpha * (gs + bs), As2 = alpha * (gs - bs);
            s.gd[o][p] = gs;
            s.nn[o][p] = ns2;
            s.pq[o][p] = valid_t ? make_float2(alpha * (gs + bs) - dvs * (1.0f - 1e-6f),
                                               alpha * (gs - bs) - dvs * (1.0f + 1e-6f))
                                 : make_float2(0.f, 0.f);
            if (a.tile_err && io >= 0 && io % kQErrEvery == 0 && valid_t && !whole) {
                // the tile's owner distance G~_cc against the FP32 and FP64 ones
                const double d64 = dist64(s.vrow[o], xrow, dim);
                if (d64 != 0.0) {
                    max_pos(&a.tile_err[0], (float)(fabs((double)gs - d64) / d64));
                    max_pos(&a.tile_err[1], (float)(fabs((double)dvs - d64) / d64));
                }
                max_pos(&a.tile_err[2], fabsf(gs - dvs) / (kappa * ns2 + 1e-30f));
                atomicAdd(&a.tile_err[3], 1u);
            }
            owner_sync(o);
            const uint64_t live = (uint64_t)s.live[o][0] | ((uint64_t)s.live[o][1] << 32);
            if (nr >= 0 && !whole) {
                // the live slots c after this lane's slot s in the order, if s is live
                const uint64_t am = valid_t ? live & ~ltm & ~(1ull << p) : 0ull;
                const float m2a = -2.0f * alpha;
                // tests the loose bound leaves open are queued and decided after the
                // loop, a lane per test (they are rare: inline, one lane's FP32
                // distance would hold up the whole warp for each)
                int nq = 0;
                for (int ch = 0; ch < 4; ++ch) {
                    const int c0 = 16 * ch;
                    const uint32_t a16 = (uint32_t)(am >> c0) & 0xffffu;
                    if (!__any_sync(0xffffffffu, a16 != 0u)) continue;   // occ stays zero
                    uint32_t rv[16];
                    tc::tmem_ld16(tl + 64 * o + c0, rv);
                    tc::tmem_wait_ld();
                    tests += (unsigned long long)__popc(a16);
                    uint32_t obits = 0;   // this lane's open tests of the chunk
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        const int c = c0 + q;
                        float g = __uint_as_float(rv[q]);
                        if (kF8) g *= isc_t * s.isc[o][c];   // exact: powers of two
                        const float2 pqc = s.pq[o][c];
                        const bool act = (a16 >> q) & 1u;
                        const float up = fmaf(m2a, g, pqc.x + As);
                        const float dn = fmaf(m2a, g, pqc.y + As2);
                        obits |= act && !(up < 0.f) && !(dn > 0.f) ? 1u << q : 0u;
                        const unsigned m = __ballot_sync(0xffffffffu, act && up < 0.f);
                        if (lane == 0) s.occ[o][c][h] = m;
                    }
                    if (__any_sync(0xffffffffu, obits != 0u)) {
                        __syncwarp();   // the occluder words above are written
                        // (the chunk's tile values again: cheaper than keeping them live)
                        tc::tmem_ld16(tl + 64 * o + c0, rv);
                        tc::tmem_wait_ld();
                        // queue slots: an exclusive prefix of the lanes' open counts
                        const int cnt = __popc(obits);
                        int pre = cnt;
#pragma unroll
                        for (int d = 1; d < 32; d <<= 1) {
                            const int t = __shfl_up_sync(0xffffffffu, pre, d);
                            if (lane >= d) pre += t;
                        }
                        int k = nq + pre - cnt;
                        nq += __shfl_sync(0xffffffffu, pre, 31);
#pragma unroll
                        for (int q = 0; q < 16; ++q) {
                            if (!((obits >> q) & 1u)) continue;
                            const int c = c0 + q;
                            float g = __uint_as_float(rv[q]);
                            if (kF8) g *= isc_t * s.isc[o][c];
                            if (k < kQOpen) {
                                s.open_q[warp][k] = make_uint2(__float_as_uint(g), (uint32_t)c | ((uint32_t)p << 8));
                            } else {   // queue full: decided here
                                const int res = decide_open(g, gs, ns2, s.gd[o][c], s.nn[o][c], s.sd[o][c],
                                                            xrow, s.rp[o][c], dim, alpha, e1, kE, gam);
                                rechecks += (unsigned long long)(res >> 1);
                                if (res & 1) atomicOr(&s.occ[o][c][h], 1u << lane);
                            }
                            ++k;
                        }
                    }
                }
                __syncwarp();
                for (int k = lane; k < min(nq, kQOpen); k += 32) {
                    const uint2 e = s.open_q[warp][k];
                    const int c = (int)(e.y & 0xffu), ps = (int)(e.y >> 8);
                    const int res = decide_open(__uint_as_float(e.x), s.gd[o][ps], s.nn[o][ps], s.gd[o][c],
                                                s.nn[o][c], s.sd[o][c], s.rp[o][ps], s.rp[o][c], dim, alpha,
                                                e1, kE, gam);
                    rechecks += (unsigned long long)(res >> 1);
                    if (res & 1) atomicOr(&s.occ[o][c][h], 1u << (ps & 31));
                }
            }
            tc::fence_before_sync();
            owner_sync(o);
            // ---- 5. the greedy walk (one warp per owner) --------------------------
            if (h == 1) {
                // meanwhile the other warp brings the rows of this warp pair's next owner
                // (same chunk) into L2
                int64_t pc = cur, nx = -1;
                for (int k = 0; k <= o; ++k) {
                    nx = -1;
                    while (pc < i1) {
                        const int64_t j = pc++;
                        int64_t cl = 0, ch = 0;
                        if (a.csr_offs) {
                            cl = a.csr_offs[j];
                            ch = a.csr_offs[j + 1];
                        }
                        if ((a.skip_empty_csr && ch == cl) || (int64_t)a.lenA + a.lenB + (ch - cl) > kQC)
                            continue;
                        nx = j;
                        break;
                    }
                }
                if (nx >= 0) {
                    const int32_t on = a.owner_ids ? a.owner_ids[nx] : (int32_t)(a.owner_base + nx);
                    const int64_t cl = a.csr_offs ? a.csr_offs[nx] : 0;
                    const int nrn = (int)((int64_t)a.lenA + a.lenB + ((a.csr_offs ? a.csr_offs[nx + 1] : 0) - cl));
                    for (int j = lane; j <= nrn; j += 32) {
                        int32_t idn = on;   // j == nrn: the owner
                        if (j < nrn) {
                            if (j < a.lenA) {
                                idn = a.listA[(int64_t)on * a.lenA + j];
                            } else if (j < a.lenA + a.lenB) {
                                idn = a.listB[nx * a.strideB + (j - a.lenA)];
                                if (idn >= 0) idn += a.offB;
                            } else {
                                idn = a.csr_ids[cl + (j - a.lenA - a.lenB)];
                            }
                        }
                        if (idn < 0) continue;
                        const char *row = reinterpret_cast<const char *>(seg_row(a.segs, idn, dim));
                        for (int l = 0; l < dim * 4; l += 128) prefetch_l2(row + l);
                    }
                }
            }
            if (nr >= 0 && h == 0) {
                // slots l and l + 32 of lane l; occluders of slot c: live slots before c
                // in the order that occlude it
                const int np = __popcll(live);
                const uint64_t lt0 = s.ltm[o][lane], lt1 = s.ltm[o][lane + 32];
                uint64_t kept = 0;
                if (a.keep_all_if_fit && np <= R) {
                    kept = live;
                } else {
                    // a slot is decided once every live occluder before it is; it is kept
                    // iff none of those is kept
                    const uint64_t oc0 =
                        ((uint64_t)s.occ[o][lane][0] | ((uint64_t)s.occ[o][lane][1] << 32)) & lt0 & live;
                    const uint64_t oc1 =
                        ((uint64_t)s.occ[o][lane + 32][0] | ((uint64_t)s.occ[o][lane + 32][1] << 32)) & lt1 & live;
                    const uint64_t b0 = 1ull << lane, b1 = 1ull << (lane + 32);
                    uint64_t decided = ~live, kall = 0ull;
                    while (~decided) {
                        const bool d0 = !(decided & b0), d1 = !(decided & b1);
                        const bool k0 = d0 && !(oc0 & kall) && !(oc0 & ~decided);
                        const bool k1 = d1 && !(oc1 & kall) && !(oc1 & ~decided);
                        const bool r0 = k0 || (d0 && (oc0 & kall));
                        const bool r1 = k1 || (d1 && (oc1 & kall));
                        decided |= (uint64_t)__ballot_sync(0xffffffffu, r0) |
                                   ((uint64_t)__ballot_sync(0xffffffffu, r1) << 32);
                        kall |= (uint64_t)__ballot_sync(0xffffffffu, k0) |
                                ((uint64_t)__ballot_sync(0xffffffffu, k1) << 32);
                    }
                    kept = kall;
                }
                // output in (distance, id) order: a kept slot's index is the number of kept
                // slots before it; the cap keeps the first R
                const int nk = min(__popcll(kept), R);
                int32_t *out = a.out + (a.out_by_index ? io : (int64_t)owner) * R;
                const int p0 = __popcll(kept & lt0), p1 = __popcll(kept & lt1);
                const bool k0 = ((kept >> lane) & 1ull) && p0 < R;
                const bool k1 = ((kept >> (lane + 32)) & 1ull) && p1 < R;
                const int32_t id0 = k0 ? (int32_t)(uint32_t)s.key[o][lane] : -1;
                const int32_t id1 = k1 ? (int32_t)(uint32_t)s.key[o][lane + 32] : -1;
                if (k0) out[p0] = id0;
                if (k1) out[p1] = id1;
                for (int j = nk + lane; j < R; j += 32) out[j] = -1;
                if (a.eu) {
                    const bool e0 = k0 && id0 >= a.emit_lo && id0 < a.emit_hi;
                    const bool e1b = k1 && id1 >= a.emit_lo && id1 < a.emit_hi;
                    const unsigned m0 = __ballot_sync(0xffffffffu, e0);
                    const unsigned m1 = __ballot_sync(0xffffffffu, e1b);
                    const int cnt = __popc(m0) + __popc(m1);
                    int base = 0;
                    if (lane == 0 && cnt) base = (int)atomicAdd(a.ecount, (unsigned long long)cnt);
                    base = __shfl_sync(0xffffffffu, base, 0);
                    if (e0) {
                        const int slot = base + __popc(m0 & lanemask_lt());
                        a.eu[slot] = id0;
                        a.ev[slot] = owner;
                    }
                    if (e1b) {
                        const int slot = base + __popc(m0) + __popc(m1 & lanemask_lt());
                        a.eu[slot] = id1;
                        a.ev[slot] = owner;
                    }
                }
            }
            tc::fence_before_sync();
            __syncthreads();   // the tile, the tensor memory and the owner state are free
            tc::fence_after_sync();
        }
        __syncthreads();   // every thread has read sh_i (and sh_fail) before the next claim
        if (sh_fail) break;
    }
    if (rechecks && a.rechecks) atomicAdd(a.rechecks, rechecks);
    if (tests && a.tile_tests) atomicAdd(a.tile_tests, tests);
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(taddr, kQCols);
}

// Order-preserving int image of a float (for atomicMin / atomicMax).
__device__ __forceinline__ int ordered(float f) {
    const int b = __float_as_int(f);
    return b >= 0 ? b : b ^ 0x7fffffff;
}

// out[0] |= 1 if a component is not an integer; out[1] / out[2]: min / max
// component (ordered ints).  blockIdx.y = segment.
__global__ void exact_range_kernel(SegTable t, int dim, int *out) {
    const int seg = blockIdx.y;
    const int64_t n4 = (t.off[seg + 1] - t.off[seg]) * dim / 4;
    const float4 *x = reinterpret_cast<const float4 *>(t.base[seg]);
    int nonint = 0;
    float lo = INFINITY, hi = -INFINITY;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n4;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float4 v = x[i];
        const float c[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            nonint |= !(c[k] == rintf(c[k]));
            lo = fminf(lo, c[k]);
            hi = fmaxf(hi, c[k]);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        nonint |= __shfl_xor_sync(0xffffffffu, nonint, o);
        lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if ((threadIdx.x & 31) == 0) {
        if (nonint) atomicOr(&out[0], 1);
        atomicMin(&out[1], ordered(lo));
        atomicMax(&out[2], ordered(hi));
    }
}

float from_ordered(int b) {
    const int v = b >= 0 ? b : b ^ 0x7fffffff;
    float f;
    memcpy(&f, &v, sizeof(f));
    return f;
}

}  // namespace

cudaError_t launch_pair_exact_check(const SegTable &t, int32_t dim, int32_t *scratch, int32_t *hi_only,
                                    cudaStream_t st) {
    *hi_only = 0;
    if (t.m <= 0 || t.off[t.m] <= 0) return cudaSuccess;
    int init[3] = {0, 0x7fffffff, (int)0x80000000};
    cudaError_t e = cudaMemcpyAsync(scratch, init, sizeof(init), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    exact_range_kernel<<<dim3(256, (unsigned)t.m), 256, 0, st>>>(t, dim, scratch);
    note_launches(1);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    int res[3];
    e = cudaMemcpyAsync(res, scratch, sizeof(res), cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return e;
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    // integers spanning at most 256: every difference of two components is an
    // integer of magnitude <= 256, exact in FP32 and in BF16 (8 significant bits)
    *hi_only = res[0] == 0 && (double)from_ordered(res[2]) - (double)from_ordered(res[1]) <= 256.0;
    return cudaSuccess;
}

bool prune_pair_ok(int dim, int prec, int metric) {
    if (metric != 0 || dim > kQMaxDim) return false;
    if (prec == 1) return dim >= 16 && dim % 16 == 0;
    return prec == 2 && dim >= 32 && dim % 32 == 0;   // E4M3: 32 elements per K-step
}

int prune_pair_max_pool() { return kQC; }

cudaError_t launch_prune_pair(const PruneArgs &in, cudaStream_t st) {
    if (!prune_pair_ok(in.dim, in.prec, in.metric) || in.R > kQC) return cudaErrorInvalidValue;
    PruneArgs a = in;
    // test-only: withhold the MMA completion signal, so every wait runs out
    a.test_withhold_commit = getenv("RNSM_TEST_WITHHOLD_COMMIT") != nullptr;
    // hi (and lo) terms, 128 rows of 2 dim bytes (BF16) or dim bytes (E4M3) each
    const bool f8 = a.prec == 2;
    const size_t dyn = (size_t)(f8 || a.pair_hi_only ? 256 : 512) * a.dim;
    auto kern = f8 ? prune_pair_kernel<2> : a.pair_hi_only ? prune_pair_kernel<1> : prune_pair_kernel<0>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    if (e != cudaSuccess) return e;
    cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, kern);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, smem_sm = 0, regs_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
    // resident CTAs per SM: shared memory (plus 1 KB reserved per CTA), registers
    // and the SM's 512 tensor-memory columns
    int per_sm = smem_sm / (int)(fa.sharedSizeBytes + dyn + 1024);
    const int by_regs = regs_sm / ((fa.numRegs > 0 ? fa.numRegs : 128) * kQT);
    if (by_regs < per_sm) per_sm = by_regs;
    if (per_sm > 512 / kQCols) per_sm = 512 / kQCols;
    if (per_sm < 1) per_sm = 1;
    // owners per claim: reverse-edge pools skip their empty owners, so they claim more,
    // but not so many that the last claims leave a tail (32: about 12 pairs)
    const int chunk = a.skip_empty_csr ? 32 : 8;
    int64_t grid = (int64_t)sms * per_sm;
    const int64_t want = (a.n_owners + chunk - 1) / chunk;
    if (want < grid) grid = want;
    kern<<<(unsigned)grid, kQT, dyn, st>>>(a, chunk);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace rnsm
