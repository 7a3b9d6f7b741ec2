// K1: batched AKNN beam search (Algorithm 1, Section 2.2), one warp per query.
//
// Per warp, in shared memory: the candidate set C as a (distance, id) array
// sorted lexicographically and double buffered (the expanded flag rides in
// bit 31 of the id), an open-addressing visited hash, and staging for the
// distances of the current neighbourhood.  Neighbour rows are gathered with
// 128-bit loads: a group of G lanes covers one row (lane s of the group reads
// float4 s, s+G, ...), 32/G rows per step, U steps in flight.
//
// Semantics match Algorithm 1 exactly: repeatedly expand the nearest
// unexpanded entry, evaluate every neighbour not evaluated before, keep the
// best ef by (distance, id).  Inserting a whole neighbourhood and truncating
// to ef leaves the same set as inserting one neighbour at a time.  The hash
// is exact until a probe sequence runs out; from then on it is lossy, which
// cannot change the result because an evaluated vertex outside C is worse
// than the worst entry of C (and that bound only tightens) while vertices
// inside C are deduplicated by id before insertion.
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
template <int VAR>
struct Variant {
    static constexpr int kUMul2 = VAR == 0 ? 1 : 2;  // rows in flight, in halves of U0
    static constexpr int kMinBlocks = VAR == 0 ? 8 : 5;
};
constexpr int kVariants = 2;

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
__device__ __forceinline__ void process(const SearchArgs &a, WarpSmem &w, int hslots,
                                        const float4 (&q)[Layout<F4>::V], int32_t c0, int32_t c1,
                                        int &size, bool &overflow, unsigned long long &ndc) {
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
            const float *row = a.base + (int64_t)(id < 0 ? 0 : id) * (4 * F4);
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

template <int F4, int EFMAX, int VAR>
__global__ void __launch_bounds__(kSearchWarps * 32, Variant<VAR>::kMinBlocks)
search_kernel(const SearchArgs a, int hslots) {
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

    unsigned long long ndc_total = 0, nexp_total = 0;
    for (;;) {
        int qi = 0;
        if (lane == 0) qi = atomicAdd(a.work, 1);
        qi = __shfl_sync(0xffffffffu, qi, 0);
        if (qi >= a.nq) break;
        const int64_t gi = a.q0 + qi;  // index in the whole batch
        const int32_t qrow = a.qidx ? a.qidx[gi] : (int32_t)gi;

        float4 q[V];
        const float *qv = a.qvecs + (int64_t)qrow * (4 * F4);
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
            const int64_t row = a.seed_row ? a.seed_row[qrow] : gi;
            const int32_t *srow = a.seed_tab + row * a.seed_stride;
            for (int s0 = 0; s0 < a.n_seeds; s0 += 64) {
                int32_t c0 = s0 + lane < a.n_seeds ? srow[s0 + lane] : -1;
                int32_t c1 = s0 + 32 + lane < a.n_seeds ? srow[s0 + 32 + lane] : -1;
                if (c0 >= a.n_base) c0 = -1;
                if (c1 >= a.n_base) c1 = -1;
                process<F4, EFMAX, VAR>(a, w, hslots, q, c0, c1, size, overflow, ndc);
            }
        } else {
            const int32_t e = a.seed_mode == kSeedSelf ? qrow : a.seed_const;
            process<F4, EFMAX, VAR>(a, w, hslots, q, lane == 0 ? e : -1, -1, size, overflow, ndc);
        }

        // Expansion loop: nearest unexpanded entry first.
        for (;;) {
            int found = -1;
            for (int b = 0; b < size; b += 32) {
                const int i = b + lane;
                const bool un = i < size && w.bi[i] >= 0;
                const unsigned m = __ballot_sync(0xffffffffu, un);
                if (m) { found = b + __ffs(m) - 1; break; }
            }
            if (found < 0) break;
            const int32_t u = w.bi[found];
            __syncwarp();
            if (lane == 0) w.bi[found] = u | kExpandedBit;
            __syncwarp();
            ++nexp;
            const int32_t *nb = a.adj + (int64_t)u * a.r_in;
            for (int j0 = 0; j0 < a.r_in; j0 += 64) {
                const int32_t c0 = j0 + lane < a.r_in ? nb[j0 + lane] : -1;
                const int32_t c1 = j0 + 32 + lane < a.r_in ? nb[j0 + 32 + lane] : -1;
                process<F4, EFMAX, VAR>(a, w, hslots, q, c0, c1, size, overflow, ndc);
            }
        }

        // Output: first k entries of C (optionally without the query vertex).
        const int32_t self = a.exclude_self ? qrow : -1;
        const int64_t orow = a.out_by_qidx ? qrow : gi;
        int32_t *oid = a.out_ids + orow * a.out_stride;
        float *od = a.out_d ? a.out_d + orow * a.out_stride : nullptr;
        int written = 0;
        for (int b = 0; b < size && written < a.k; b += 32) {
            const int i = b + lane;
            const int32_t id = i < size ? (w.bi[i] & kIdMask) : -1;
            const bool keep = i < size && id != self;
            const unsigned m = __ballot_sync(0xffffffffu, keep);
            const int pos = written + __popc(m & lanemask_lt());
            if (keep && pos < a.k) {
                oid[pos] = id + a.id_offset;
                if (od) od[pos] = w.bd[i];
            }
            written += __popc(m);
        }
        for (int j = written + lane; j < a.k; j += 32) {
            oid[j] = -1;
            if (od) od[j] = FLT_MAX;
        }
        if (lane == 0 && a.out_ndc) a.out_ndc[gi] = (int64_t)ndc;
        ndc_total += ndc;
        nexp_total += nexp;
        __syncwarp();
    }
    if (lane == 0 && a.stats) {
        atomicAdd(&a.stats[0], ndc_total);
        atomicAdd(&a.stats[1], nexp_total);
    }
}

int hslots_for(int ef) {
    // NDC runs at ~13-20 per beam entry on degree-32 graphs: 24 slots per
    // entry keep the load factor near 0.6 (at least 1024, a multiple of 32)
    int h = 24 * ef;
    if (h < 1024) h = 1024;
    return (h + 31) & ~31;
}

template <int F4, int EFMAX, int VAR>
cudaError_t launch_t(const SearchArgs &a, cudaStream_t st) {
    const int hslots = hslots_for(a.ef);
    const size_t smem = (size_t)kSearchWarps * warp_smem_bytes(EFMAX, hslots);
    auto kern = search_kernel<F4, EFMAX, VAR>;
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
    kern<<<(unsigned)grid, kSearchWarps * 32, smem, st>>>(a, hslots);
    note_launches(1);
    return cudaGetLastError();
}

template <int F4, int EFMAX>
cudaError_t launch_var(const SearchArgs &a, int var, cudaStream_t st) {
    return var == 0 ? launch_t<F4, EFMAX, 0>(a, st) : launch_t<F4, EFMAX, 1>(a, st);
}

template <int F4>
cudaError_t launch_ef(const SearchArgs &a, int var, cudaStream_t st) {
    if (a.ef <= 32) return launch_var<F4, 32>(a, var, st);
    if (a.ef <= 64) return launch_var<F4, 64>(a, var, st);
    if (a.ef <= 128) return launch_var<F4, 128>(a, var, st);
    return launch_var<F4, 256>(a, var, st);
}

cudaError_t launch_dim(const SearchArgs &a, int var, cudaStream_t st) {
    switch (a.dim) {
        case 8: return launch_ef<2>(a, var, st);
        case 16: return launch_ef<4>(a, var, st);
        case 32: return launch_ef<8>(a, var, st);
        case 64: return launch_ef<16>(a, var, st);
        case 96: return launch_ef<24>(a, var, st);
        case 128: return launch_ef<32>(a, var, st);
        case 256: return launch_ef<64>(a, var, st);
        case 768: return launch_ef<192>(a, var, st);
        default: return cudaErrorInvalidValue;
    }
}

// The queries [q0, q1) of a launch as a launch of their own.
SearchArgs subrange(const SearchArgs &a, int64_t q0, int64_t q1) {
    SearchArgs b = a;
    b.q0 = a.q0 + q0;
    b.nq = q1 - q0;
    return b;
}

// Autotuner: the first launch with at least kTuneMin queries for a (dim,
// beam) shape runs every variant on slices of its queries: one untimed
// warm-up slice each, then two timed slices each in alternating order (CUDA
// events on the launching stream); the variant with the smallest time per
// slice is kept for later launches.  Every variant computes the same results,
// so the choice never changes them.
constexpr int64_t kTuneWarm = 2000;
constexpr int64_t kTuneSlice = 10000;
constexpr int64_t kTuneMin = kVariants * (kTuneWarm + 2 * kTuneSlice) + 10000;
std::mutex g_tune_mu;
std::map<std::pair<int, int>, int> g_tuned;

int efmax_of(int ef) { return ef <= 32 ? 32 : ef <= 64 ? 64 : ef <= 128 ? 128 : 256; }

}  // namespace

int search_variant_for(int dim, int ef) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tuned.find({dim, efmax_of(ef)});
    return it == g_tuned.end() ? -1 : it->second;
}

namespace {

}  // namespace

cudaError_t launch_search(const SearchArgs &a, cudaStream_t st) {
    if (a.nq <= 0) return cudaSuccess;
    if (!search_dim_supported(a.dim)) return cudaErrorInvalidValue;
    const char *force = getenv("RNSM_SEARCH_VARIANT");
    if (force && (force[0] == '0' || force[0] == '1')) return launch_dim(a, force[0] - '0', st);
    const std::pair<int, int> key{a.dim, efmax_of(a.ef)};
    int var = -1;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tuned.find(key);
        if (it != g_tuned.end()) var = it->second;
    }
    if (var >= 0 || a.nq < kTuneMin) return launch_dim(a, var >= 0 ? var : 0, st);
    // slices of the batch run in turn; their results are final
    float best_ms[kVariants];
    for (int v = 0; v < kVariants; ++v) best_ms[v] = 3.4e38f;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return launch_dim(a, 0, st);
    cudaError_t err = cudaSuccess;
    int64_t pos = 0;
    auto run_slice = [&](int v, int64_t len, bool timed) {
        const SearchArgs sl = subrange(a, pos, pos + len);
        pos += len;
        err = cudaMemsetAsync(a.work, 0, sizeof(int32_t), st);  // each slice starts its own count
        if (err != cudaSuccess) return;
        if (timed) cudaEventRecord(e0, st);
        err = launch_dim(sl, v, st);
        if (err != cudaSuccess || !timed) return;
        cudaEventRecord(e1, st);
        err = cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best_ms[v]) best_ms[v] = ms;
    };
    for (int v = 0; v < kVariants && err == cudaSuccess; ++v) run_slice(v, kTuneWarm, false);
    for (int rep = 0; rep < 2 && err == cudaSuccess; ++rep)
        for (int k = 0; k < kVariants && err == cudaSuccess; ++k)
            run_slice(rep == 0 ? k : kVariants - 1 - k, kTuneSlice, true);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err != cudaSuccess) return err;
    int best = 0;
    for (int v = 1; v < kVariants; ++v)
        if (best_ms[v] < best_ms[best]) best = v;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tuned[key] = best;
    }
    err = cudaMemsetAsync(a.work, 0, sizeof(int32_t), st);
    if (err != cudaSuccess) return err;
    return launch_dim(subrange(a, pos, a.nq), best, st);
}

bool search_dim_supported(int dim) {
    switch (dim) {
        case 8: case 16: case 32: case 64: case 96: case 128: case 256: case 768: return true;
        default: return false;
    }
}

}  // namespace rnsm
