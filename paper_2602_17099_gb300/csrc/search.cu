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

#include "internal.h"

namespace rnsm {

namespace {

constexpr int kSearchWarps = 4;
constexpr int kProbes = 12;
constexpr int kCandMax = 64;   // candidates evaluated per batch

// Beam buffer c (0 or 1) holds EFMAX distances then EFMAX ids at
// beam + c * 2 * EFMAX words; indexing by arithmetic keeps it out of local memory.
struct WarpSmem {
    float *beam;
    int efmax;
    int32_t *hash;
    float *cd;
    int32_t *ci;
    float *sd;
    int32_t *si;
    __device__ __forceinline__ float *bd(int c) const { return beam + c * 2 * efmax; }
    __device__ __forceinline__ int32_t *bi(int c) const {
        return reinterpret_cast<int32_t *>(beam + c * 2 * efmax + efmax);
    }
};

__host__ __device__ constexpr size_t warp_smem_bytes(int efmax, int hbits) {
    return (size_t)efmax * 16 + ((size_t)4 << hbits) + kCandMax * 8 + 32 * 8;
}

template <int F4>
struct Layout {
    static constexpr int quarter = F4 / 4 > 0 ? F4 / 4 : 1;
    static constexpr int G = quarter >= 32 ? 32 : quarter >= 16 ? 16 : quarter >= 8 ? 8
                           : quarter >= 4 ? 4 : quarter >= 2 ? 2 : 1;
    static constexpr int V = (F4 + G - 1) / G;   // float4 per lane per row
    static constexpr int RPI = 32 / G;            // rows per step
    static constexpr int U = V <= 4 ? 8 / V : 2;  // steps in flight
};

__device__ __forceinline__ bool hash_insert(int32_t *hash, int hbits, int32_t id, bool &overflow) {
    const uint32_t hmask = (1u << hbits) - 1u;
    uint32_t h = ((uint32_t)id * 0x9E3779B1u) >> (32 - hbits);
#pragma unroll 1
    for (int p = 0; p < kProbes; ++p) {
        uint32_t slot = (h + p) & hmask;
        int32_t old = atomicCAS(&hash[slot], -1, id);
        if (old == -1) return true;
        if (old == id) return false;
    }
    overflow = true;  // treated as unseen; results stay exact (see header)
    return true;
}

// Evaluates up to 64 candidate ids (two per lane: c0 = list[lane],
// c1 = list[32 + lane]) and merges the new ones into C.
template <int F4>
__device__ __forceinline__ void process(const SearchArgs &a, WarpSmem &w, int hbits,
                                        const float4 (&q)[Layout<F4>::V], int32_t c0, int32_t c1,
                                        int &cur, int &size, bool &overflow,
                                        unsigned long long &ndc) {
    using Lay = Layout<F4>;
    constexpr int G = Lay::G, V = Lay::V, RPI = Lay::RPI, U = Lay::U;
    const int lane = threadIdx.x & 31;
    const int grp = lane / G, sub = lane % G;
    const int ef = a.ef;

    bool ovf = false;
    bool n0 = c0 >= 0 && hash_insert(w.hash, hbits, c0, ovf);
    bool n1 = c1 >= 0 && hash_insert(w.hash, hbits, c1, ovf);
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

    // Merge, 32 candidates at a time.
    for (int b0 = 0; b0 < c; b0 += 32) {
        const int j = b0 + lane;
        float d = INFINITY;
        int32_t id = INT32_MAX;
        bool valid = j < c;
        if (valid) {
            d = w.cd[j];
            id = w.ci[j];
        }
        if (valid && size == ef)
            valid = lex_less(d, id, w.bd(cur)[ef - 1], w.bi(cur)[ef - 1] & kIdMask);
        if (valid && overflow) {
            for (int i = 0; i < size; ++i)
                if ((w.bi(cur)[i] & kIdMask) == id) { valid = false; break; }
        }
        if (!valid) { d = INFINITY; id = INT32_MAX; }
        // +inf distances never enter C: keep the sentinel strictly last
        warp_sort32(d, id);
        const int32_t pid = __shfl_up_sync(0xffffffffu, id, 1);
        const bool keep = id != INT32_MAX && !(lane > 0 && pid == id);
        const unsigned km = __ballot_sync(0xffffffffu, keep);
        const int mm = __popc(km);
        if (keep) {
            const int rk = __popc(km & lanemask_lt());
            w.sd[rk] = d;
            w.si[rk] = id;
        }
        __syncwarp();
        if (mm == 0) continue;
        const int nxt = cur ^ 1;
        for (int i = lane; i < size; i += 32) {
            const float od = w.bd(cur)[i];
            const int32_t oi = w.bi(cur)[i];
            const int pos = i + lower_bound_lex(w.sd, w.si, mm, od, oi & kIdMask);
            if (pos < ef) { w.bd(nxt)[pos] = od; w.bi(nxt)[pos] = oi; }
        }
        if (lane < mm) {
            const float nd = w.sd[lane];
            const int32_t ni = w.si[lane];
            const int pos = lane + lower_bound_lex(w.bd(cur), w.bi(cur), size, nd, ni);
            if (pos < ef) { w.bd(nxt)[pos] = nd; w.bi(nxt)[pos] = ni; }
        }
        __syncwarp();
        cur = nxt;
        size = min(ef, size + mm);
    }
}

template <int F4, int EFMAX>
__global__ void __launch_bounds__(kSearchWarps * 32)
search_kernel(const SearchArgs a, int hbits) {
    using Lay = Layout<F4>;
    constexpr int G = Lay::G, V = Lay::V;
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    unsigned char *base = smem + (size_t)warp * warp_smem_bytes(EFMAX, hbits);
    WarpSmem w;
    w.beam = reinterpret_cast<float *>(base);
    w.efmax = EFMAX;
    w.hash = reinterpret_cast<int32_t *>(w.beam + 4 * EFMAX);
    w.cd = reinterpret_cast<float *>(w.hash + (1 << hbits));
    w.ci = reinterpret_cast<int32_t *>(w.cd + kCandMax);
    w.sd = reinterpret_cast<float *>(w.ci + kCandMax);
    w.si = reinterpret_cast<int32_t *>(w.sd + 32);
    const int H = 1 << hbits;
    const int sub = lane % G;

    unsigned long long ndc_total = 0, nexp_total = 0;
    for (;;) {
        int qi = 0;
        if (lane == 0) qi = atomicAdd(a.work, 1);
        qi = __shfl_sync(0xffffffffu, qi, 0);
        if (qi >= a.nq) break;
        const int32_t qrow = a.qidx ? a.qidx[qi] : qi;

        float4 q[V];
        const float *qv = a.qvecs + (int64_t)qrow * (4 * F4);
#pragma unroll
        for (int j = 0; j < V; ++j) {
            const int f = sub + G * j;
            q[j] = f < F4 ? ldg4(qv + 4 * f) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        for (int i = lane; i < H; i += 32) w.hash[i] = -1;
        __syncwarp();

        int cur = 0, size = 0;
        bool overflow = false;
        unsigned long long ndc = 0, nexp = 0;

        // Entry points.
        if (a.seed_mode == kSeedTable) {
            const int64_t row = a.seed_row ? a.seed_row[qrow] : qi;
            const int32_t *srow = a.seed_tab + row * a.seed_stride;
            for (int s0 = 0; s0 < a.n_seeds; s0 += 64) {
                int32_t c0 = s0 + lane < a.n_seeds ? srow[s0 + lane] : -1;
                int32_t c1 = s0 + 32 + lane < a.n_seeds ? srow[s0 + 32 + lane] : -1;
                if (c0 >= a.n_base) c0 = -1;
                if (c1 >= a.n_base) c1 = -1;
                process<F4>(a, w, hbits, q, c0, c1, cur, size, overflow, ndc);
            }
        } else {
            const int32_t e = a.seed_mode == kSeedSelf ? qrow : a.seed_const;
            process<F4>(a, w, hbits, q, lane == 0 ? e : -1, -1, cur, size, overflow, ndc);
        }

        // Expansion loop: nearest unexpanded entry first.
        for (;;) {
            int found = -1;
            for (int b = 0; b < size; b += 32) {
                const int i = b + lane;
                const bool un = i < size && w.bi(cur)[i] >= 0;
                const unsigned m = __ballot_sync(0xffffffffu, un);
                if (m) { found = b + __ffs(m) - 1; break; }
            }
            if (found < 0) break;
            const int32_t u = w.bi(cur)[found];
            __syncwarp();
            if (lane == 0) w.bi(cur)[found] = u | kExpandedBit;
            __syncwarp();
            ++nexp;
            const int32_t *nb = a.adj + (int64_t)u * a.r_in;
            for (int j0 = 0; j0 < a.r_in; j0 += 64) {
                const int32_t c0 = j0 + lane < a.r_in ? nb[j0 + lane] : -1;
                const int32_t c1 = j0 + 32 + lane < a.r_in ? nb[j0 + 32 + lane] : -1;
                process<F4>(a, w, hbits, q, c0, c1, cur, size, overflow, ndc);
            }
        }

        // Output: first k entries of C (optionally without the query vertex).
        const int32_t self = a.exclude_self ? qrow : -1;
        const int64_t orow = a.out_by_qidx ? qrow : qi;
        int32_t *oid = a.out_ids + orow * a.out_stride;
        float *od = a.out_d ? a.out_d + orow * a.out_stride : nullptr;
        int written = 0;
        for (int b = 0; b < size && written < a.k; b += 32) {
            const int i = b + lane;
            const int32_t id = i < size ? (w.bi(cur)[i] & kIdMask) : -1;
            const bool keep = i < size && id != self;
            const unsigned m = __ballot_sync(0xffffffffu, keep);
            const int pos = written + __popc(m & lanemask_lt());
            if (keep && pos < a.k) {
                oid[pos] = id + a.id_offset;
                if (od) od[pos] = w.bd(cur)[i];
            }
            written += __popc(m);
        }
        for (int j = written + lane; j < a.k; j += 32) {
            oid[j] = -1;
            if (od) od[j] = FLT_MAX;
        }
        if (lane == 0 && a.out_ndc) a.out_ndc[qi] = (int64_t)ndc;
        ndc_total += ndc;
        nexp_total += nexp;
        __syncwarp();
    }
    if (lane == 0 && a.stats) {
        atomicAdd(&a.stats[0], ndc_total);
        atomicAdd(&a.stats[1], nexp_total);
    }
}

int hbits_for(int ef) {
    // NDC runs at ~15-20 per beam entry on degree-32 graphs: 32 slots per
    // entry keep the load factor near 0.5 (at least 1024, at most 8192 slots)
    int h = 10;
    while ((1 << h) < 32 * ef && h < 13) ++h;
    return h;
}

template <int F4, int EFMAX>
cudaError_t launch_t(const SearchArgs &a, cudaStream_t st) {
    const int hbits = hbits_for(a.ef);
    const size_t smem = (size_t)kSearchWarps * warp_smem_bytes(EFMAX, hbits);
    auto kern = search_kernel<F4, EFMAX>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    // the visited hashes live in shared memory: ask for the largest carveout
    cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kSearchWarps * 32, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    int64_t want = (a.nq + kSearchWarps - 1) / kSearchWarps;
    int64_t grid = (int64_t)sms * per_sm;
    if (want < grid) grid = want < 1 ? 1 : want;
    kern<<<(unsigned)grid, kSearchWarps * 32, smem, st>>>(a, hbits);
    note_launches(1);
    return cudaGetLastError();
}

template <int F4>
cudaError_t launch_ef(const SearchArgs &a, cudaStream_t st) {
    if (a.ef <= 32) return launch_t<F4, 32>(a, st);
    if (a.ef <= 64) return launch_t<F4, 64>(a, st);
    if (a.ef <= 128) return launch_t<F4, 128>(a, st);
    return launch_t<F4, 256>(a, st);
}

}  // namespace

cudaError_t launch_search(const SearchArgs &a, cudaStream_t st) {
    if (a.nq <= 0) return cudaSuccess;
    switch (a.dim) {
        case 8: return launch_ef<2>(a, st);
        case 16: return launch_ef<4>(a, st);
        case 32: return launch_ef<8>(a, st);
        case 64: return launch_ef<16>(a, st);
        case 96: return launch_ef<24>(a, st);
        case 128: return launch_ef<32>(a, st);
        case 256: return launch_ef<64>(a, st);
        case 768: return launch_ef<192>(a, st);
        default: return cudaErrorInvalidValue;
    }
}

bool search_dim_supported(int dim) {
    switch (dim) {
        case 8: case 16: case 32: case 64: case 96: case 128: case 256: case 768: return true;
        default: return false;
    }
}

}  // namespace rnsm
