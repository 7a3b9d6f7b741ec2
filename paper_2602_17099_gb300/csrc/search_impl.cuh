// Kernel templates and launchers of K1, the batched beam search; included by
// the two translation units that instantiate them (single-job launches in
// search.cu, multi-job launches in search_jobs.cu, compiled in parallel).
#pragma once
#include <float.h>
#include <stdlib.h>

#include <map>
#include <mutex>
#include <utility>

#include "internal.h"

namespace rnsm {

namespace {

constexpr int kSearchWarps = 4;
constexpr int kProbes = 12;
constexpr int kCandMax = 64;   // candidates evaluated per batch

// The candidate set C: EFMAX distances, then EFMAX ids (expanded flag in bit 31).
struct WarpSmem {
    float *bd;
    int32_t *bi;
    int32_t *hash;
    float *cd;
    int32_t *ci;
    float *sd;
    int32_t *si;
};

__host__ __device__ constexpr size_t warp_smem_bytes(int efmax, int hslots) {
    return (size_t)efmax * 8 + (size_t)4 * hslots + kCandMax * 16;
}

// Launch-shape variants (identical results): 0 = half the rows in flight and
// registers capped for 8 CTAs per SM; 1 = the full rows in flight, 5 CTAs.
// A tuned variant number v selects shape v & 1 and, if v & 2, the L2
// prefetch of the runner-up's neighbourhood during each expansion.
template <int VAR>
struct Variant {
    static constexpr int kUMul2 = VAR == 0 ? 1 : 2;  // rows in flight, in halves of U0
    static constexpr int kMinBlocks = VAR == 0 ? 8 : 5;
};
constexpr int kVariants = 4;

template <int F4, int UMUL2 = 2>
struct Layout {
    static constexpr int quarter = F4 / 4 > 0 ? F4 / 4 : 1;
    static constexpr int G = quarter >= 32 ? 32 : quarter >= 16 ? 16 : quarter >= 8 ? 8
                           : quarter >= 4 ? 4 : quarter >= 2 ? 2 : 1;
    static constexpr int V = (F4 + G - 1) / G;   // float4 per lane per row
    static constexpr int RPI = 32 / G;            // rows per step
    static constexpr int U0 = V <= 4 ? 8 / V : 2;
    static constexpr int U = U0 * UMUL2 / 2 > 0 ? U0 * UMUL2 / 2 : 1;  // steps in flight
};

// Open addressing over H slots (any H): multiply-shift start, linear probing.
__device__ __forceinline__ bool hash_insert(int32_t *hash, int H, int32_t id, bool &overflow) {
    uint32_t slot = (uint32_t)(((uint64_t)((uint32_t)id * 0x9E3779B1u) * (uint32_t)H) >> 32);
#pragma unroll 1
    for (int p = 0; p < kProbes; ++p) {
        int32_t old = atomicCAS(&hash[slot], -1, id);
        if (old == -1) return true;
        if (old == id) return false;
        slot = slot + 1 == (uint32_t)H ? 0u : slot + 1;
    }
    overflow = true;  // treated as unseen; results stay exact (see header)
    return true;
}

// Evaluates up to 64 candidate ids (two per lane: c0 = list[lane],
// c1 = list[32 + lane]) and merges the new ones into C.
template <int F4, int EFMAX, int VAR>
__device__ __forceinline__ void process(const SearchArgs &a, const float *base, WarpSmem &w, int hslots,
                                        const float4 (&q)[Layout<F4>::V], int32_t c0, int32_t c1,
                                        int &size, bool &overflow, unsigned long long &ndc,
                                        int32_t pf = -1) {
    using Lay = Layout<F4, Variant<VAR>::kUMul2>;
    constexpr int G = Lay::G, V = Lay::V, RPI = Lay::RPI, U = Lay::U;
    const int lane = threadIdx.x & 31;
    const int grp = lane / G, sub = lane % G;
    const int ef = a.ef;

    bool ovf = false;
    bool n0 = c0 >= 0 && hash_insert(w.hash, hslots, c0, ovf);
    bool n1 = c1 >= 0 && hash_insert(w.hash, hslots, c1, ovf);
    if (__any_sync(0xffffffffu, ovf)) overflow = true;
    unsigned m0 = __ballot_sync(0xffffffffu, n0);
    unsigned m1 = __ballot_sync(0xffffffffu, n1);
    const int cnt0 = __popc(m0);
    const int c = cnt0 + __popc(m1);
    if (n0) w.ci[__popc(m0 & lanemask_lt())] = c0;
    if (n1) w.ci[cnt0 + __popc(m1 & lanemask_lt())] = c1;
    // pf: a neighbour of the entry likely to be expanded next; its row is brought
    // into L2 now so that the next expansion's gather finds it there (a hint only)
    if (pf >= 0) {
        const char *pr = reinterpret_cast<const char *>(base + (int64_t)pf * (4 * F4));
#pragma unroll
        for (int l = 0; l < 16 * F4; l += 128) prefetch_l2(pr + l);
    }
    __syncwarp();
    if (c == 0) return;
    ndc += (unsigned long long)c;

    // Distances of the new candidates.
    for (int b0 = 0; b0 < c; b0 += RPI * U) {
        float4 x[U][V];
        int rr[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int r = b0 + u * RPI + grp;
            rr[u] = r;
            const int32_t id = r < c ? w.ci[r] : -1;
            const float *row = base + (int64_t)(id < 0 ? 0 : id) * (4 * F4);
#pragma unroll
            for (int j = 0; j < V; ++j) {
                const int f = sub + G * j;
                x[u][j] = (id >= 0 && f < F4) ? ldg4(row + 4 * f) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            float acc = 0.f;
            if (a.metric == 0) {
#pragma unroll
                for (int j = 0; j < V; ++j)
                    if (sub + G * j < F4) acc = l2_acc(acc, q[j], x[u][j]);
            } else {
#pragma unroll
                for (int j = 0; j < V; ++j)
                    if (sub + G * j < F4) acc = ip_acc(acc, q[j], x[u][j]);
            }
#pragma unroll
            for (int off = G / 2; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
            if (sub == 0 && rr[u] < c) w.cd[rr[u]] = a.metric == 0 ? acc : 1.0f - acc;
        }
    }
    __syncwarp();

    // Survivors: candidates that beat the worst entry of a full C (and, after
    // a hash overflow, are not in C already), compacted into (sd, si).
    int m = 0;
    for (int b0 = 0; b0 < c; b0 += 32) {
        const int j = b0 + lane;
        float d = INFINITY;
        int32_t id = INT32_MAX;
        bool keep = j < c;
        if (keep) {
            d = w.cd[j];
            id = w.ci[j];
        }
        if (keep && size == ef) keep = lex_less(d, id, w.bd[ef - 1], w.bi[ef - 1] & kIdMask);
        if (keep && overflow) {
            for (int i = 0; i < size; ++i)
                if ((w.bi[i] & kIdMask) == id) { keep = false; break; }
            for (int i = 0; keep && i < b0 + lane; ++i)   // a lossy hash can repeat an id
                if (w.ci[i] == id) keep = false;
        }
        const unsigned km = __ballot_sync(0xffffffffu, keep);
        if (keep) {
            const int rk = m + __popc(km & lanemask_lt());
            w.sd[rk] = d;
            w.si[rk] = id;
        }
        m += __popc(km);
    }
    __syncwarp();
    if (m == 0) return;
    // Merge by ranks, in place: old entry i moves to i + #{new < it}; new entry
    // k goes to #{new < it} + #{old < it}; entries past ef fall off.
    constexpr int PER = EFMAX / 32;
    float od[PER];
    int32_t oi[PER];
    int sh[PER];
#pragma unroll
    for (int t = 0; t < PER; ++t) {
        const int i = lane + 32 * t;
        od[t] = i < size ? w.bd[i] : INFINITY;
        oi[t] = i < size ? w.bi[i] : INT32_MAX;
        sh[t] = 0;
    }
    const float nd0 = lane < m ? w.sd[lane] : INFINITY;
    const int32_t ni0 = lane < m ? w.si[lane] : INT32_MAX;
    const float nd1 = lane + 32 < m ? w.sd[lane + 32] : INFINITY;
    const int32_t ni1 = lane + 32 < m ? w.si[lane + 32] : INT32_MAX;
    int r0 = 0, r1 = 0;
    for (int k = 0; k < m; ++k) {
        const float dk = w.sd[k];
        const int32_t ik = w.si[k];
        r0 += lex_less(dk, ik, nd0, ni0);
        r1 += lex_less(dk, ik, nd1, ni1);
#pragma unroll
        for (int t = 0; t < PER; ++t) sh[t] += lex_less(dk, ik, od[t], oi[t] & kIdMask);
    }
    if (lane < m) r0 += lower_bound_lex(w.bd, w.bi, size, nd0, ni0);
    if (lane + 32 < m) r1 += lower_bound_lex(w.bd, w.bi, size, nd1, ni1);
    __syncwarp();
#pragma unroll
    for (int t = 0; t < PER; ++t) {
        const int i = lane + 32 * t;
        const int pos = i + sh[t];
        if (i < size && pos < ef) { w.bd[pos] = od[t]; w.bi[pos] = oi[t]; }
    }
    if (lane < m && r0 < ef) { w.bd[r0] = nd0; w.bi[r0] = ni0; }
    if (lane + 32 < m && r1 < ef) { w.bd[r1] = nd1; w.bi[r1] = ni1; }
    __syncwarp();
    size = min(ef, size + m);
}

// JOBS: query g of the launch belongs to the job j with
// jobs[j].q_begin <= g < jobs[j + 1].q_begin and is query g - q_begin of that
// job; the job's fields replace the launch's (one launch, many pairs).
#define JF(f) (JOBS ? J->f : a.f)

template <int F4, int EFMAX, int VAR, bool JOBS>
__global__ void __launch_bounds__(kSearchWarps * 32, Variant<VAR>::kMinBlocks)
search_kernel(const SearchArgs a, int hslots, int prefetch) {
    using Lay = Layout<F4>;
    constexpr int G = Lay::G, V = Lay::V;
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    unsigned char *base = smem + (size_t)warp * warp_smem_bytes(EFMAX, hslots);
    WarpSmem w;
    w.bd = reinterpret_cast<float *>(base);
    w.bi = reinterpret_cast<int32_t *>(w.bd + EFMAX);
    w.hash = w.bi + EFMAX;
    w.cd = reinterpret_cast<float *>(w.hash + hslots);
    w.ci = reinterpret_cast<int32_t *>(w.cd + kCandMax);
    w.sd = reinterpret_cast<float *>(w.ci + kCandMax);
    w.si = reinterpret_cast<int32_t *>(w.sd + kCandMax);
    const int H = hslots;
    const int sub = lane % G;
    __shared__ SearchJob sjob[JOBS ? kSearchWarps : 1];

    unsigned long long ndc_total = 0, nexp_total = 0;
    for (;;) {
        int qi = 0;
        if (lane == 0) qi = atomicAdd(a.work, 1);
        qi = __shfl_sync(0xffffffffu, qi, 0);
        if (qi >= a.nq) break;
        int64_t gi = a.q0 + qi;  // index in the whole batch (JOBS: in its job)
        const SearchJob *J = nullptr;
        if (JOBS) {
            int lo = 0, hi = a.n_jobs - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (a.jobs[mid].q_begin <= gi) lo = mid; else hi = mid - 1;
            }
            // the job's fields go to this warp's shared slot and are read from
            // there when needed (no registers held across the query)
            static_assert(sizeof(SearchJob) % 4 == 0 && sizeof(SearchJob) <= 128, "job copy");
            const int32_t *src = reinterpret_cast<const int32_t *>(a.jobs + lo);
            int32_t *dst = reinterpret_cast<int32_t *>(&sjob[warp]);
            if (lane < (int)(sizeof(SearchJob) / 4)) dst[lane] = src[lane];
            __syncwarp();
            J = &sjob[warp];
            gi -= J->q_begin;
        }
        const float *base = JF(base);
        const int32_t *qidx = JF(qidx);
        const int32_t qrow = qidx ? qidx[gi] : (int32_t)gi;

        float4 q[V];
        const float *qv = JF(qvecs) + (int64_t)qrow * (4 * F4);
#pragma unroll
        for (int j = 0; j < V; ++j) {
            const int f = sub + G * j;
            q[j] = f < F4 ? ldg4(qv + 4 * f) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        for (int i = lane; i < H; i += 32) w.hash[i] = -1;
        __syncwarp();

        int size = 0;
        bool overflow = false;
        unsigned long long ndc = 0, nexp = 0;

        // Entry points.
        if (a.seed_mode == kSeedTable) {
            const int32_t *seed_row = JF(seed_row);
            const int64_t n_base = JF(n_base);
            const int64_t row = seed_row ? seed_row[qrow] : gi;
            const int32_t *srow = JF(seed_tab) + row * a.seed_stride;
            for (int s0 = 0; s0 < a.n_seeds; s0 += 64) {
                int32_t c0 = s0 + lane < a.n_seeds ? srow[s0 + lane] : -1;
                int32_t c1 = s0 + 32 + lane < a.n_seeds ? srow[s0 + 32 + lane] : -1;
                if (c0 >= n_base) c0 = -1;
                if (c1 >= n_base) c1 = -1;
                process<F4, EFMAX, VAR>(a, base, w, hslots, q, c0, c1, size, overflow, ndc);
            }
        } else {
            const int32_t e = a.seed_mode == kSeedSelf ? qrow : JF(seed_const);
            process<F4, EFMAX, VAR>(a, base, w, hslots, q, lane == 0 ? e : -1, -1, size, overflow, ndc);
        }

        // Expansion loop: nearest unexpanded entry first.
        for (;;) {
            // the nearest unexpanded entry and the runner-up (usually expanded next)
            int found = -1, second = -1;
            for (int b = 0; b < size && (prefetch ? second < 0 : found < 0); b += 32) {
                const int i = b + lane;
                const bool un = i < size && w.bi[i] >= 0;
                unsigned m = __ballot_sync(0xffffffffu, un);
                if (found < 0 && m) {
                    found = b + __ffs(m) - 1;
                    m &= m - 1u;
                }
                if (found >= 0 && m) second = b + __ffs(m) - 1;
            }
            if (found < 0) break;
            const int32_t u = w.bi[found];
            const int r_in = JF(r_in);
            const int32_t *adj = JF(adj);
            // one neighbour of the runner-up per lane, to prefetch during this expansion
            int32_t pf = -1;
            if (prefetch && second >= 0 && lane < r_in) pf = adj[(int64_t)(w.bi[second] & kIdMask) * r_in + lane];
            __syncwarp();
            if (lane == 0) w.bi[found] = u | kExpandedBit;
            __syncwarp();
            ++nexp;
            const int32_t *nb = adj + (int64_t)u * r_in;
            for (int j0 = 0; j0 < r_in; j0 += 64) {
                const int32_t c0 = j0 + lane < r_in ? nb[j0 + lane] : -1;
                const int32_t c1 = j0 + 32 + lane < r_in ? nb[j0 + 32 + lane] : -1;
                process<F4, EFMAX, VAR>(a, base, w, hslots, q, c0, c1, size, overflow, ndc,
                                        j0 == 0 ? pf : -1);
            }
        }

        // Output: first k entries of C (optionally without the query vertex).
        const int32_t self = a.exclude_self ? qrow : -1;
        const int64_t orow = a.out_by_qidx ? qrow : gi;
        int32_t *oid = JF(out_ids) + orow * a.out_stride;
        float *od = (!JOBS && a.out_d) ? a.out_d + orow * a.out_stride : nullptr;
        const int32_t id_offset = JF(id_offset);
        int written = 0;
        for (int b = 0; b < size && written < a.k; b += 32) {
            const int i = b + lane;
            const int32_t id = i < size ? (w.bi[i] & kIdMask) : -1;
            const bool keep = i < size && id != self;
            const unsigned m = __ballot_sync(0xffffffffu, keep);
            const int pos = written + __popc(m & lanemask_lt());
            if (keep && pos < a.k) {
                oid[pos] = id + id_offset;
                if (od) od[pos] = w.bd[i];
            }
            written += __popc(m);
        }
        for (int j = written + lane; j < a.k; j += 32) {
            oid[j] = -1;
            if (od) od[j] = FLT_MAX;
        }
        if (!JOBS && lane == 0 && a.out_ndc) a.out_ndc[gi] = (int64_t)ndc;
        ndc_total += ndc;
        nexp_total += nexp;
        __syncwarp();
    }
    if (lane == 0 && a.stats) {
        atomicAdd(&a.stats[0], ndc_total);
        atomicAdd(&a.stats[1], nexp_total);
    }
}

#undef JF

int hslots_for(int ef) {
    // NDC runs at ~13-20 per beam entry on degree-32 graphs: 24 slots per
    // entry keep the load factor near 0.6 (at least 1024, a multiple of 32)
    int h = 24 * ef;
    if (h < 1024) h = 1024;
    return (h + 31) & ~31;
}

template <int F4, int EFMAX, int VAR, bool JOBS>
cudaError_t launch_t(const SearchArgs &a, int prefetch, cudaStream_t st) {
    const int hslots = hslots_for(a.ef);
    const size_t smem = (size_t)kSearchWarps * warp_smem_bytes(EFMAX, hslots);
    auto kern = search_kernel<F4, EFMAX, VAR, JOBS>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    // the visited hashes live in shared memory: ask for the largest carveout
    cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, kern);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, smem_sm = 0, regs_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
    int per_sm = smem_sm / (int)(fa.sharedSizeBytes + smem + 1024);
    const int by_regs = regs_sm / ((fa.numRegs > 0 ? fa.numRegs : 64) * kSearchWarps * 32);
    if (by_regs < per_sm) per_sm = by_regs;
    if (per_sm > 2048 / (kSearchWarps * 32)) per_sm = 2048 / (kSearchWarps * 32);
    if (per_sm < 1) per_sm = 1;
    int64_t want = (a.nq + kSearchWarps - 1) / kSearchWarps;
    int64_t grid = (int64_t)sms * per_sm;
    if (want < grid) grid = want < 1 ? 1 : want;
    kern<<<(unsigned)grid, kSearchWarps * 32, smem, st>>>(a, hslots, prefetch);
    note_launches(1);
    return cudaGetLastError();
}

template <int F4, int EFMAX, bool JOBS>
cudaError_t launch_var(const SearchArgs &a, int var, cudaStream_t st) {
    const int pf = (var >> 1) & 1;
    return (var & 1) == 0 ? launch_t<F4, EFMAX, 0, JOBS>(a, pf, st) : launch_t<F4, EFMAX, 1, JOBS>(a, pf, st);
}

template <int F4, bool JOBS>
cudaError_t launch_ef(const SearchArgs &a, int var, cudaStream_t st) {
    if (a.ef <= 32) return launch_var<F4, 32, JOBS>(a, var, st);
    if (a.ef <= 64) return launch_var<F4, 64, JOBS>(a, var, st);
    if (a.ef <= 128) return launch_var<F4, 128, JOBS>(a, var, st);
    return launch_var<F4, 256, JOBS>(a, var, st);
}

template <bool JOBS>
cudaError_t launch_dim(const SearchArgs &a, int var, cudaStream_t st) {
    switch (a.dim) {
        case 8: return launch_ef<2, JOBS>(a, var, st);
        case 16: return launch_ef<4, JOBS>(a, var, st);
        case 32: return launch_ef<8, JOBS>(a, var, st);
        case 64: return launch_ef<16, JOBS>(a, var, st);
        case 96: return launch_ef<24, JOBS>(a, var, st);
        case 128: return launch_ef<32, JOBS>(a, var, st);
        case 256: return launch_ef<64, JOBS>(a, var, st);
        case 768: return launch_ef<192, JOBS>(a, var, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace
}  // namespace rnsm
