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

__device__ __forceinline__ float4 ldg4(const float *p) {
    return __ldg(reinterpret_cast<const float4 *>(p));
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
