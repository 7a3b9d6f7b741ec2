// K2 on the tensor cores: the small-pool occlusion prune with the
// candidate-by-candidate distance tile computed as a BF16 or FP8 (E4M3,
// per-row scale) Gram matrix by tcgen05.mma with FP32 accumulation in tensor
// memory, and every decision the low-precision tile cannot settle re-decided
// with the exact FP32 distance.  The result equals the FP32 prune's.
//
// Per owner: the quantized owner row and up to 64 candidate rows are staged
// in shared memory in the K-major no-swizzle layout; one thread issues the
// MMAs (M = 128 rows, N = 80 columns), commits them to an mbarrier, and every
// warp reads its 32 TMEM lanes.  From the Gram entries G the tile holds
//   L2: d~(i,j) = G_ii + G_jj - 2 G_ij,   IP: d~(i,j) = 1 - G_ij,
// and a bound B(i,j) >= |d~(i,j) - d(i,j)| where d is the FP32 prune's value
// (the fixed FP32 chain over the dimensions): quantisation error from the
// rows' residual norms e = ||x - x~||, the FP32 accumulation error of the
// Gram, and the chain's own rounding.  A candidate whose owner-distance
// interval overlaps another's gets its exact FP32 owner distance, so the
// candidate order equals the FP32 order; an occlusion test whose interval
// for alpha*d(s,c) - d(v,c) contains zero is recomputed in FP32 and decided
// with the same fmaf(alpha, d(s,c), -d(v,c)) <= 0.
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <float.h>

#include "internal.h"
#include "tcgen05.cuh"

namespace rnsm {

namespace {

constexpr int kThreads = 128;
constexpr int kMax = 64;          // raw pool entries
constexpr int kRows = kMax + 1;   // owner + candidates
constexpr int kM = 128;           // MMA rows (rows past kRows are never read back)
constexpr int kN = 80;            // MMA columns: kRows rounded up to 16
constexpr int kTmemCols = 128;
constexpr long kSpinLimit = 1L << 26;

__device__ __forceinline__ int tri(int a, int b, int n) { return a * (2 * n - a - 1) / 2 + (b - a - 1); }

// The FP32 prune's distance: one fmaf chain over the dimensions in order
// (loads issued eight float4 ahead; the arithmetic order is unchanged).
__device__ float exact_dist(const float *a, const float *b, int dim, int metric) {
    float acc = 0.f;
    const int F4 = dim >> 2;
    int f = 0;
    for (; f + 8 <= F4; f += 8) {
        float4 x[8], y[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            x[u] = ldg4(a + 4 * (f + u));
            y[u] = ldg4(b + 4 * (f + u));
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) acc = metric == 0 ? l2_acc(acc, x[u], y[u]) : ip_acc(acc, x[u], y[u]);
    }
    for (; f < F4; ++f) {
        const float4 x = ldg4(a + 4 * f), y = ldg4(b + 4 * f);
        acc = metric == 0 ? l2_acc(acc, x, y) : ip_acc(acc, x, y);
    }
    return metric == 0 ? acc : 1.0f - acc;
}

constexpr int kPairs = kRows * (kRows - 1) / 2;

struct TcSmem {
    float Gd[kRows];          // scaled Gram diagonal
    float e[kRows];           // residual norms of the stored quantisation
    float ep[kRows];          // residual norms of the per-tile re-quantisation (L2)
    float sc[kRows];          // per-row scale of the staged tile row
    float nr[kRows];          // row norms
    int32_t pid[kMax];
    const float *rptr[kRows];
    float dx[kMax];            // exact owner distance (valid if ex[c])
    int32_t ex[kMax];
    float kd[kMax];
    int32_t kix[kMax];
    float sd[kMax];
    int32_t sid[kMax];
    int32_t srow[kMax];
    uint32_t occ[2 * kMax];
    int32_t need_ex[kMax];
    float res[kRows];          // staging reductions (L2)
    float dsum[kRows];
    uint32_t mx[kRows];
    int n_undecided;
    uint64_t bar;
    uint32_t tmem_slot;
};

template <bool kFp8>
__global__ void __launch_bounds__(kThreads) prune_tc_kernel(const PruneArgs a, int chunk) {
    extern __shared__ __align__(1024) unsigned char tile[];   // quantized rows, K-major no swizzle
    __shared__ TcSmem s;
    __shared__ int64_t sh_i;
    __shared__ int sh_fail;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int dim = a.dim;
    const int R = a.R;
    const int metric = a.metric;
    const int esz = kFp8 ? 1 : 2;
    const int row_bytes = dim * esz;
    const int chunks = row_bytes / 16;
    const uint32_t LBO = 128, SBO = (uint32_t)chunks * 128;
    const int ksteps = row_bytes / 32;   // 16 BF16 or 32 E4M3 per MMA
    const float eps_c = kFp8 ? (float)dim * 9.5367431640625e-07f  // 2^-20 per term
                             : (float)dim * 2.384185791e-07f;     // 2^-22 per term
    const float gam = (float)(dim + 4) * 1.1920929e-07f;           // FP32 chain, 2^-23 per term
    const unsigned char *Q = static_cast<const unsigned char *>(a.qrows);

    if (tid == 0) {
        tc::mbar_init(&s.bar, 1);
        sh_fail = 0;
    }
    if (warp == 0) {
        tc::tmem_alloc(&s.tmem_slot, kTmemCols);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = s.tmem_slot;
    const uint32_t tbase = tc::smem_u32(tile);
    // Once an owner's MMA has completed its staged rows are dead: the tile
    // buffer then holds the d~ triangle, the bound triangle and the list of
    // undecided tests ((s << 16) | c).
    float *const T = reinterpret_cast<float *>(tile);
    float *const Bt = T + kPairs;
    uint32_t *const undecided = reinterpret_cast<uint32_t *>(Bt + kPairs);
    uint32_t phase = 0;
    unsigned long long rechecks = 0;

    for (;;) {
        if (tid == 0) sh_i = atomicAdd(a.work, chunk);
        __syncthreads();
        const int64_t i0 = sh_i;
        if (i0 >= a.n_owners || sh_fail) break;
        const int64_t i1 = min(a.n_owners, i0 + chunk);
      for (int64_t i = i0; i < i1; ++i) {
        const int32_t owner = a.owner_ids ? a.owner_ids[i] : (int32_t)(a.owner_base + i);
        int64_t c_lo = 0, c_hi = 0;
        if (a.csr_offs) {
            c_lo = a.csr_offs[i];
            c_hi = a.csr_offs[i + 1];
        }
        if (a.skip_empty_csr && c_hi == c_lo) continue;
        const int64_t nr_raw = (int64_t)a.lenA + a.lenB + (c_hi - c_lo);
        if (nr_raw > kMax) {
            if (tid == 0) a.ovf_list[atomicAdd(a.ovf_count, 1ull)] = (int32_t)i;
            continue;
        }
        const int nr = (int)nr_raw, nrows = 1 + nr;
        // 1. pool ids (the owner and -1 become -1) and row metadata
        for (int j = tid; j < kMax; j += kThreads) {
            int32_t id = -1;
            if (j < nr) {
                if (j < a.lenA) {
                    id = a.listA[(int64_t)owner * a.lenA + j];
                } else if (j < a.lenA + a.lenB) {
                    id = a.listB[i * a.strideB + (j - a.lenA)];
                    if (id >= 0) id += a.offB;
                } else {
                    id = a.csr_ids[c_lo + (j - a.lenA - a.lenB)];
                }
                if (id == owner) id = -1;
            }
            s.pid[j] = id;
        }
        __syncthreads();
        for (int r = tid; r < nrows; r += kThreads) {
            const int32_t g = r == 0 ? owner : (s.pid[r - 1] >= 0 ? s.pid[r - 1] : owner);
            s.e[r] = a.qerr[g];
            s.nr[r] = a.qnorm[g];
            s.rptr[r] = seg_row(a.segs, g, dim);
        }
        // 2. stage the tile rows.  L2: every row is re-centred on the owner
        //    (x~_r - x~_v, re-quantised), so the Gram entries are of the size of
        //    the distances themselves and the tile is free of cancellation;
        //    integer-valued data stays exact.  IP: the stored rows as they are.
        if (metric == 0) {
            for (int r = tid; r < nrows; r += kThreads) {
                s.res[r] = 0.f;
                s.dsum[r] = 0.f;
                s.mx[r] = 0u;
            }
            __syncthreads();
            if (kFp8) {  // per-row scale of the centred row: max |x~_r - x~_v| / 448
                for (int e = tid; e < nrows * chunks; e += kThreads) {
                    const int r = e / chunks, j = e - r * chunks;
                    const int32_t g = r == 0 ? owner : (s.pid[r - 1] >= 0 ? s.pid[r - 1] : owner);
                    const uint4 av = *reinterpret_cast<const uint4 *>(Q + (int64_t)g * row_bytes + 16 * j);
                    const uint4 ov = *reinterpret_cast<const uint4 *>(Q + (int64_t)owner * row_bytes + 16 * j);
                    const __nv_fp8_e4m3 *ab = reinterpret_cast<const __nv_fp8_e4m3 *>(&av);
                    const __nv_fp8_e4m3 *ob = reinterpret_cast<const __nv_fp8_e4m3 *>(&ov);
                    const float sg = a.qscale[g], so = a.qscale[owner];
                    float m = 0.f;
#pragma unroll
                    for (int k = 0; k < 16; ++k)
                        m = fmaxf(m, fabsf(sg * static_cast<float>(ab[k]) - so * static_cast<float>(ob[k])));
                    atomicMax(&s.mx[r], __float_as_uint(m));
                }
                __syncthreads();
            }
            for (int e = tid; e < nrows * chunks; e += kThreads) {
                const int r = e / chunks, j = e - r * chunks;
                const int32_t g = r == 0 ? owner : (s.pid[r - 1] >= 0 ? s.pid[r - 1] : owner);
                const uint4 av = *reinterpret_cast<const uint4 *>(Q + (int64_t)g * row_bytes + 16 * j);
                const uint4 ov = *reinterpret_cast<const uint4 *>(Q + (int64_t)owner * row_bytes + 16 * j);
                float res = 0.f, dsum = 0.f;
                uint4 outv;
                if (kFp8) {
                    const __nv_fp8_e4m3 *ab = reinterpret_cast<const __nv_fp8_e4m3 *>(&av);
                    const __nv_fp8_e4m3 *ob = reinterpret_cast<const __nv_fp8_e4m3 *>(&ov);
                    const float sg = a.qscale[g], so = a.qscale[owner];
                    const float mxr = __uint_as_float(s.mx[r]);
                    const float scale = mxr > 0.f ? mxr / 448.0f : 1.0f;
                    unsigned char *ob8 = reinterpret_cast<unsigned char *>(&outv);
#pragma unroll
                    for (int k = 0; k < 16; ++k) {
                        const float dlt = sg * static_cast<float>(ab[k]) - so * static_cast<float>(ob[k]);
                        const __nv_fp8_e4m3 q(dlt / scale);
                        const float rr = dlt - scale * static_cast<float>(q);
                        res = fmaf(rr, rr, res);
                        dsum = fmaf(dlt, dlt, dsum);
                        ob8[k] = *reinterpret_cast<const unsigned char *>(&q);
                    }
                } else {
                    const __nv_bfloat16 *ab = reinterpret_cast<const __nv_bfloat16 *>(&av);
                    const __nv_bfloat16 *ob = reinterpret_cast<const __nv_bfloat16 *>(&ov);
                    __nv_bfloat16 *qo = reinterpret_cast<__nv_bfloat16 *>(&outv);
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        const float dlt = __bfloat162float(ab[k]) - __bfloat162float(ob[k]);
                        qo[k] = __float2bfloat16_rn(dlt);
                        const float rr = dlt - __bfloat162float(qo[k]);
                        res = fmaf(rr, rr, res);
                        dsum = fmaf(dlt, dlt, dsum);
                    }
                }
                *reinterpret_cast<uint4 *>(tile + (r >> 3) * SBO + j * LBO + (r & 7) * 16) = outv;
                if (res > 0.f) atomicAdd(&s.res[r], res);
                if (dsum > 0.f) atomicAdd(&s.dsum[r], dsum);
            }
            __syncthreads();
            for (int r = tid; r < nrows; r += kThreads) {
                // re-quantisation residual (rounded up: the atomic sum's order varies),
                // plus the rounding of the FP32 subtraction
                const float res = s.res[r];
                s.ep[r] = (res > 0.f ? sqrtf(res) * 1.001f : 0.f) + 2.4e-7f * sqrtf(s.dsum[r]);
                const float mxr = __uint_as_float(s.mx[r]);
                s.sc[r] = kFp8 ? (mxr > 0.f ? mxr / 448.0f : 1.0f) : 1.0f;
            }
        } else {
            for (int e = tid; e < nrows * chunks; e += kThreads) {
                const int r = e / chunks, j = e - r * chunks;
                const int32_t g = r == 0 ? owner : (s.pid[r - 1] >= 0 ? s.pid[r - 1] : owner);
                const uint4 v = *reinterpret_cast<const uint4 *>(Q + (int64_t)g * row_bytes + 16 * j);
                *reinterpret_cast<uint4 *>(tile + (r >> 3) * SBO + j * LBO + (r & 7) * 16) = v;
            }
            for (int r = tid; r < nrows; r += kThreads) {
                const int32_t g = r == 0 ? owner : (s.pid[r - 1] >= 0 ? s.pid[r - 1] : owner);
                s.ep[r] = 0.f;
                s.sc[r] = kFp8 ? a.qscale[g] : 1.f;
            }
        }
        tc::fence_async_shared();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        // 3. the Gram tile on the tensor cores
        if (tid == 0) {
            const uint32_t idesc = tc::instr_desc(kFp8 ? 0u : 1u, kM, kN);
            for (int k = 0; k < ksteps; ++k) {
                const uint64_t d = tc::smem_desc(tbase + k * 2 * LBO, LBO, SBO);
                if (kFp8) tc::mma_fp8(taddr, d, d, idesc, k > 0);
                else tc::mma_bf16(taddr, d, d, idesc, k > 0);
            }
            tc::mma_commit(&s.bar);
        }
        bool ok = true;
        for (long it = 0; !tc::mbar_try_wait(&s.bar, phase); ++it)
            if (it > kSpinLimit) { ok = false; break; }
        const int timed_out = __syncthreads_or(!ok);   // one decision for the whole CTA
        phase ^= 1u;
        if (timed_out) {
            if (tid == 0) { atomicOr(a.err, 64); sh_fail = 1; }
            break;
        }
        tc::fence_after_sync();
        // 4. epilogue: diagonal first, then the triangle with its bounds
        const int row = 32 * warp + lane;
        const float srow_scale = row < nrows ? s.sc[row] : 1.f;
        if (warp < 3) {
            for (int c = 0; c < kN / 16; ++c) {
                uint32_t r[16];
                tc::tmem_ld16(taddr + ((uint32_t)(32 * warp) << 16) + 16 * c, r);
                tc::tmem_wait_ld();
                if (row < nrows && row >= 16 * c && row < 16 * c + 16)
                    s.Gd[row] = __uint_as_float(r[row - 16 * c]) * srow_scale * srow_scale;
            }
        }
        __syncthreads();
        if (warp < 3) {
            for (int c = 0; c < kN / 16; ++c) {
                uint32_t r[16];
                tc::tmem_ld16(taddr + ((uint32_t)(32 * warp) << 16) + 16 * c, r);
                tc::tmem_wait_ld();
                if (row < nrows) {
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        const int col = 16 * c + q;
                        if (col <= row || col >= nrows) continue;
                        const float g = __uint_as_float(r[q]) * srow_scale * s.sc[col];
                        const float gi = s.Gd[row], gj = s.Gd[col];
                        const float E = s.e[row] + s.e[col] + s.ep[row] + s.ep[col];
                        float dt, bq, bc, bf;
                        if (metric == 0) {
                            dt = gi + gj - 2.0f * g;
                            bc = eps_c * (gi + gj + 2.0f * fabsf(g));
                            const float t = sqrtf(fmaxf(dt + bc, 0.f));
                            bq = 2.0f * t * E + 3.0f * E * E;
                            bf = gam * (fmaxf(dt, 0.f) + bq + bc);
                        } else {
                            dt = 1.0f - g;
                            bc = eps_c * sqrtf(fmaxf(gi, 0.f) * fmaxf(gj, 0.f));
                            bq = s.nr[row] * s.e[col] + s.e[row] * s.nr[col] + s.e[row] * s.e[col];
                            bf = gam * s.nr[row] * s.nr[col] + 1.2e-7f;
                        }
                        const int t = tri(row, col, nrows);
                        T[t] = dt;
                        Bt[t] = 1.01f * (bq + bc + bf) + 1e-30f;
                    }
                }
            }
        }
        tc::fence_before_sync();
        __syncthreads();
        // 5. owner distances: exact where the intervals of two candidates overlap
        for (int c = tid; c < kMax; c += kThreads) {
            s.ex[c] = 0;
            if (c < nr && s.pid[c] >= 0) {
                const float dc = T[tri(0, 1 + c, nrows)], bc = Bt[tri(0, 1 + c, nrows)];
                bool clash = false;
                for (int k = 0; k < nr && !clash; ++k) {
                    if (k == c || s.pid[k] < 0) continue;
                    const float dk = T[tri(0, 1 + k, nrows)], bk = Bt[tri(0, 1 + k, nrows)];
                    clash = fabsf(dc - dk) <= (bc + bk) * 1.0001f;
                }
                if (clash) {
                    s.dx[c] = exact_dist(s.rptr[0], s.rptr[1 + c], dim, metric);
                    s.ex[c] = 1;
                    ++rechecks;
                }
            }
        }
        __syncthreads();
        // 6. order by (distance, id): exact keys where resolved, else the tile's
        for (int j = tid; j < kMax; j += kThreads) {
            const bool valid = j < nr && s.pid[j] >= 0;
            s.kd[j] = valid ? (s.ex[j] ? s.dx[j] : T[tri(0, 1 + j, nrows)]) : INFINITY;
            s.kix[j] = valid ? s.pid[j] : INT32_MAX;
        }
        __syncthreads();
        for (int j = tid; j < nr; j += kThreads) {
            const float dj = s.kd[j];
            const int32_t ij = s.kix[j];
            int r = 0;
            for (int k = 0; k < nr; ++k) {
                const float dk = s.kd[k];
                const int32_t ik = s.kix[k];
                r += lex_less(dk, ik, dj, ij) || (dk == dj && ik == ij && k < j);
            }
            s.sd[r] = dj;
            s.sid[r] = ij;
            s.srow[r] = 1 + j;
        }
        __syncthreads();
        // 7. occluder masks.  Pass 1 settles what the tile can and lists the
        //    rest; pass 2 computes the missing exact owner distances; pass 3
        //    recomputes every listed test in FP32, one test per thread.
        if (tid == 0) s.n_undecided = 0;
        for (int c = tid; c < kMax; c += kThreads) s.need_ex[c] = 0;
        __syncthreads();
        for (int c = warp; c < nr; c += kThreads / 32) {
            const int cr = s.srow[c];
            const bool cvalid = s.sid[c] != INT32_MAX;
            const bool cex = cvalid && s.ex[cr - 1];
            const float dvc = s.sd[c];
            const float bvc = cex ? 0.f : (cvalid ? Bt[tri(0, cr, nrows)] : 0.f);
            bool t[2] = {false, false};
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int sp = lane + 32 * h;
                if (sp >= c || s.sid[sp] == INT32_MAX || !cvalid) continue;
                const int sr = s.srow[sp];
                const int tt = sr < cr ? tri(sr, cr, nrows) : tri(cr, sr, nrows);
                const float dsc = T[tt], bsc = Bt[tt];
                const float lo = a.alpha * (dsc - bsc) - (dvc + bvc);
                const float hi = a.alpha * (dsc + bsc) - (dvc - bvc);
                const float slack = 1e-6f * (a.alpha * (fabsf(dsc) + bsc) + fabsf(dvc) + bvc);
                if (hi + slack < 0.f) {
                    t[h] = true;
                } else if (!(lo - slack > 0.f)) {
                    undecided[atomicAdd(&s.n_undecided, 1)] = ((uint32_t)sp << 16) | (uint32_t)c;
                    if (!cex) s.need_ex[cr - 1] = 1;
                }
            }
            const unsigned m0 = __ballot_sync(0xffffffffu, t[0]);
            const unsigned m1 = __ballot_sync(0xffffffffu, t[1]);
            if (lane == 0) {
                s.occ[2 * c] = m0;
                s.occ[2 * c + 1] = m1;
            }
        }
        __syncthreads();
        for (int j = tid; j < nr; j += kThreads) {
            if (s.need_ex[j] && !s.ex[j]) {
                s.dx[j] = exact_dist(s.rptr[0], s.rptr[1 + j], dim, metric);
                s.ex[j] = 1;
                ++rechecks;
            }
        }
        __syncthreads();
        const int nu = s.n_undecided;
        for (int u = tid; u < nu; u += kThreads) {
            const uint32_t code = undecided[u];
            const int sp = (int)(code >> 16), c = (int)(code & 0xffffu);
            const int sr = s.srow[sp], cr = s.srow[c];
            const float xs = exact_dist(s.rptr[sr], s.rptr[cr], dim, metric);
            const float xv = s.ex[cr - 1] ? s.dx[cr - 1] : s.sd[c];
            if (fmaf(a.alpha, xs, -xv) <= 0.f) atomicOr(&s.occ[2 * c + (sp >> 5)], 1u << (sp & 31));
            ++rechecks;
        }
        __syncthreads();
        // 8. greedy walk and output (as the FP32 small-pool prune)
        if (warp == 0) {
            const bool a0 = lane < nr && s.sid[lane] != INT32_MAX &&
                            (lane == 0 || s.sid[lane - 1] != s.sid[lane]);
            const bool a1 = lane + 32 < nr && s.sid[lane + 32] != INT32_MAX &&
                            s.sid[lane + 31] != s.sid[lane + 32];
            const unsigned long long live = (unsigned long long)__ballot_sync(0xffffffffu, a0) |
                                            ((unsigned long long)__ballot_sync(0xffffffffu, a1) << 32);
            const int np = __popcll(live);
            unsigned long long kept = 0;
            int nk = 0;
            if (a.keep_all_if_fit && np <= R) {
                kept = live;
                nk = np;
            } else {
                for (int c = 0; c < nr && nk < R; ++c) {
                    if (!((live >> c) & 1ull)) continue;
                    const unsigned long long oc = (unsigned long long)s.occ[2 * c] |
                                                  ((unsigned long long)s.occ[2 * c + 1] << 32);
                    if (!(oc & kept)) {
                        kept |= 1ull << c;
                        ++nk;
                    }
                }
            }
            int32_t *out = a.out + (a.out_by_index ? i : (int64_t)owner) * R;
            const bool k0 = (kept >> lane) & 1ull, k1 = (kept >> (lane + 32)) & 1ull;
            const int p0 = __popcll(kept & ((1ull << lane) - 1ull));
            const int p1 = __popcll(kept & ((1ull << (lane + 32)) - 1ull));
            const int32_t id0 = k0 ? s.sid[lane] : -1, id1 = k1 ? s.sid[lane + 32] : -1;
            if (k0) out[p0] = id0;
            if (k1) out[p1] = id1;
            for (int j = nk + lane; j < R; j += 32) out[j] = -1;
            if (a.eu) {
                const bool e0 = k0 && id0 >= a.emit_lo && id0 < a.emit_hi;
                const bool e1 = k1 && id1 >= a.emit_lo && id1 < a.emit_hi;
                const unsigned b0 = __ballot_sync(0xffffffffu, e0);
                const unsigned b1 = __ballot_sync(0xffffffffu, e1);
                const int cnt = __popc(b0) + __popc(b1);
                int base = 0;
                if (lane == 0 && cnt) base = (int)atomicAdd(a.ecount, (unsigned long long)cnt);
                base = __shfl_sync(0xffffffffu, base, 0);
                if (e0) {
                    const int slot = base + __popc(b0 & lanemask_lt());
                    a.eu[slot] = id0;
                    a.ev[slot] = owner;
                }
                if (e1) {
                    const int slot = base + __popc(b0) + __popc(b1 & lanemask_lt());
                    a.eu[slot] = id1;
                    a.ev[slot] = owner;
                }
            }
        }
        tc::fence_before_sync();
        __syncthreads();
      }
        __syncthreads();  // every thread has read sh_i (and sh_fail) before the next claim
        tc::fence_after_sync();
        if (sh_fail) break;
    }
    if (rechecks && a.rechecks) atomicAdd(a.rechecks, rechecks);
    if (sh_fail) {  // give an MMA that did not finish a second bounded chance before freeing TMEM
        for (long it = 0; !tc::mbar_try_wait(&s.bar, phase ^ 1u) && it < kSpinLimit; ++it) {
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(taddr, kTmemCols);
}

// Row quantisation: BF16 (round to nearest) or E4M3 with a per-row scale
// (max |x| / 448), the residual norm ||x - x~|| (rounded up) and ||x||.
template <bool kFp8>
__global__ void quantize_kernel(SegTable segs, int64_t n, int32_t dim, void *q, float *scale,
                                float *err, float *norm) {
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = w0; r < n; r += nw) {
        const float *x = seg_row(segs, (int32_t)r, dim);
        float mx = 0.f, nn = 0.f;
        for (int k = lane; k < dim; k += 32) {
            const float v = x[k];
            mx = fmaxf(mx, fabsf(v));
            nn = fmaf(v, v, nn);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            nn += __shfl_xor_sync(0xffffffffu, nn, o);
        }
        const float sc = kFp8 ? (mx > 0.f ? mx / 448.0f : 1.0f) : 1.0f;
        float ee = 0.f;
        for (int k = lane; k < dim; k += 32) {
            const float v = x[k];
            float back;
            if (kFp8) {
                const __nv_fp8_e4m3 t(v / sc);
                reinterpret_cast<__nv_fp8_e4m3 *>(q)[r * dim + k] = t;
                back = sc * static_cast<float>(t);
            } else {
                const __nv_bfloat16 t = __float2bfloat16_rn(v);
                reinterpret_cast<__nv_bfloat16 *>(q)[r * dim + k] = t;
                back = __bfloat162float(t);
            }
            const float dlt = v - back;
            ee = fmaf(dlt, dlt, ee);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) ee += __shfl_xor_sync(0xffffffffu, ee, o);
        if (lane == 0) {
            if (kFp8) scale[r] = sc;
            err[r] = ee > 0.f ? sqrtf(ee) * 1.001f + 1e-30f : 0.f;
            norm[r] = sqrtf(nn) * 1.0001f;
        }
    }
}

}  // namespace

bool prune_tc_supported(int dim, int prec) {
    if (prec != 1 && prec != 2) return false;
    const int row_bytes = dim * (prec == 2 ? 1 : 2);
    return row_bytes % 32 == 0 && (size_t)kM * row_bytes <= 64 * 1024;
}

cudaError_t launch_prune_tc(const PruneArgs &a, cudaStream_t st) {
    const bool fp8 = a.prec == 2;
    size_t dyn = (size_t)kM * a.dim * (fp8 ? 1 : 2);
    const size_t after = (size_t)kPairs * 12;   // triangles + undecided list
    if (dyn < after) dyn = after;
    auto kern = fp8 ? prune_tc_kernel<true> : prune_tc_kernel<false>;
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
    // resident CTAs per SM: shared memory (plus 1 KB reserved per CTA), registers,
    // and the SM's 512 tensor-memory columns (kTmemCols per CTA)
    int per_sm = smem_sm / (int)(fa.sharedSizeBytes + dyn + 1024);
    const int by_regs = regs_sm / ((fa.numRegs > 0 ? fa.numRegs : 64) * kThreads);
    if (by_regs < per_sm) per_sm = by_regs;
    if (per_sm > 512 / kTmemCols) per_sm = 512 / kTmemCols;
    if (per_sm < 1) per_sm = 1;
    const int chunk = a.skip_empty_csr ? 32 : 1;
    int64_t grid = (int64_t)sms * per_sm;
    const int64_t want = (a.n_owners + chunk - 1) / chunk;
    if (want < grid) grid = want;
    kern<<<(unsigned)grid, kThreads, dyn, st>>>(a, chunk);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_quantize(const SegTable &segs, int64_t n, int32_t dim, int prec, void *q,
                            float *scale, float *err, float *norm, cudaStream_t st) {
    int64_t g = (n * 32 + 255) / 256;
    if (g > 16384) g = 16384;
    if (g < 1) g = 1;
    if (prec == 2) quantize_kernel<true><<<(unsigned)g, 256, 0, st>>>(segs, n, dim, q, scale, err, norm);
    else quantize_kernel<false><<<(unsigned)g, 256, 0, st>>>(segs, n, dim, q, scale, err, norm);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace rnsm
