// Device helpers shared by the RNSM kernels (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace rnsm {

constexpr int kWarp = 32;
constexpr int kMaxSeg = 64;          // segments addressable by one merge
constexpr int32_t kExpandedBit = int32_t(0x80000000u);
constexpr int32_t kIdMask = 0x7fffffff;

// Global id -> row pointer over up to kMaxSeg separately allocated segments.
struct SegTable {
    const float *base[kMaxSeg];
    int64_t off[kMaxSeg + 1];
    int32_t m;
};

__device__ __forceinline__ const float *seg_row(const SegTable &t, int32_t gid, int dim) {
    int lo = 0, hi = t.m - 1;
    while (lo < hi) {  // last segment with off <= gid
        int mid = (lo + hi + 1) >> 1;
        if (t.off[mid] <= gid) lo = mid; else hi = mid - 1;
    }
    return t.base[lo] + (int64_t)(gid - t.off[lo]) * dim;
}

// Lexicographic (distance, id) order; ties to the lower id.
__device__ __forceinline__ bool lex_less(float da, int32_t ia, float db, int32_t ib) {
    return da < db || (da == db && ia < ib);
}

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Ascending bitonic sort of one (d, id) pair per lane across the warp.
__device__ __forceinline__ void warp_sort32(float &d, int32_t &id) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            float od = __shfl_xor_sync(0xffffffffu, d, j);
            int32_t oi = __shfl_xor_sync(0xffffffffu, id, j);
            bool up = (lane & k) == 0;
            bool lower = (lane & j) == 0;
            // the lower lane of a pair keeps the min when ascending, the max otherwise
            bool take = (lower == up) ? lex_less(od, oi, d, id) : lex_less(d, id, od, oi);
            if (take) { d = od; id = oi; }
        }
    }
}

// Number of entries of sorted (sd, si)[0..n) that are lex-less than (d, id).
__device__ __forceinline__ int lower_bound_lex(const float *sd, const int32_t *si, int n,
                                               float d, int32_t id) {
    int lo = 0, hi = n;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (lex_less(sd[mid], si[mid] & kIdMask, d, id)) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ void prefetch_l2(const void *p) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

__device__ __forceinline__ float4 ldg4(const float *p) {
    return __ldg(reinterpret_cast<const float4 *>(p));
}

// ---- the FP32 prune distance ---------------------------------------------
// One definition for every kernel that takes an occlusion decision: two
// chains over the dimensions, E over the even ones and O over the odd ones,
// each acc = fmaf(a_k - b_k, a_k - b_k, acc) (L2) or fmaf(a_k, b_k, acc) (IP)
// in increasing k; then d = E + O (L2) or 1 - (E + O) (IP).  Both chains of a
// pair live in one 64-bit register (low half E) and advance together in one
// packed f32x2 instruction, whose lanes round exactly as the scalar ones.
typedef unsigned long long f2_t;

__device__ __forceinline__ f2_t f2_of(float lo, float hi) {
    f2_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void f2_split(f2_t a, float &lo, float &hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(a));
}
__device__ __forceinline__ f2_t f2_sub(f2_t a, f2_t b) {
    f2_t r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2_t f2_fma(f2_t a, f2_t b, f2_t c) {
    f2_t r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}
// Four consecutive dimensions (two f32x2 halves) of rows a and b.
__device__ __forceinline__ f2_t chain2(f2_t acc, ulonglong2 a, ulonglong2 b, int metric) {
    if (metric == 0) {
        const f2_t d0 = f2_sub(a.x, b.x);
        acc = f2_fma(d0, d0, acc);
        const f2_t d1 = f2_sub(a.y, b.y);
        return f2_fma(d1, d1, acc);
    }
    acc = f2_fma(a.x, b.x, acc);
    return f2_fma(a.y, b.y, acc);
}
__device__ __forceinline__ float chain2_final(f2_t acc, int metric) {
    float e, o;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(e), "=f"(o) : "l"(acc));
    const float s = e + o;
    return metric == 0 ? s : 1.0f - s;
}
__device__ __forceinline__ ulonglong2 ldg_u2(const float *p) {
    return __ldg(reinterpret_cast<const ulonglong2 *>(p));
}
// d(a, b) over dim (a multiple of 4) dimensions from global memory.
__device__ __forceinline__ float prune_dist(const float *a, const float *b, int dim, int metric) {
    f2_t acc = 0ull;
    const int F4 = dim >> 2;
    int f = 0;
    for (; f + 8 <= F4; f += 8) {   // loads issued eight ahead of their use
        ulonglong2 x[8], y[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            x[u] = ldg_u2(a + 4 * (f + u));
            y[u] = ldg_u2(b + 4 * (f + u));
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) acc = chain2(acc, x[u], y[u], metric);
    }
    for (; f < F4; ++f) acc = chain2(acc, ldg_u2(a + 4 * f), ldg_u2(b + 4 * f), metric);
    return chain2_final(acc, metric);
}

__device__ __forceinline__ float l2_acc(float acc, float4 q, float4 x) {
    float a = q.x - x.x, b = q.y - x.y, c = q.z - x.z, e = q.w - x.w;
    acc = fmaf(a, a, acc);
    acc = fmaf(b, b, acc);
    acc = fmaf(c, c, acc);
    acc = fmaf(e, e, acc);
    return acc;
}

__device__ __forceinline__ float ip_acc(float acc, float4 q, float4 x) {
    acc = fmaf(q.x, x.x, acc);
    acc = fmaf(q.y, x.y, acc);
    acc = fmaf(q.z, x.z, acc);
    acc = fmaf(q.w, x.w, acc);
    return acc;
}

}  // namespace rnsm
