// Query schedule of the batched searches (S1, S4, S5): the order in which
// the warps take their queries.  Every query is independent, so any order
// gives the same results; an order in which consecutive queries lie close
// together lets the warps that run side by side share vector rows and
// adjacency rows in L2 instead of fetching them from HBM one query at a time.
//
// Locality key: nb <= 12 random hyperplanes, hyperplane j through a data
// point of the segment; bit j of a vertex's key is the side it lies on.  The
// vertices of a segment are counting-sorted by key (order, used by S1) and
// each gets its position in that order (rank).  After S3 the pivots are
// sorted by rank (S4) and the followers by the rank of their pivot (S5), so a
// pivot's followers are adjacent and nearby pivots are searched together.
#include <stdint.h>

#include "internal.h"

namespace rnsm {

namespace {

constexpr int kMaxPlanes = 12;

// Entry k of hyperplane j: a uniform value in [-1, 1) from an integer hash.
__device__ __forceinline__ float plane_entry(uint32_t j, uint32_t k) {
    uint32_t h = j * 0x9E3779B1u + k * 0x85EBCA77u + 0x165667B1u;
    h ^= h >> 15;
    h *= 0x2C1B3C6Du;
    h ^= h >> 12;
    h *= 0x297A2D39u;
    h ^= h >> 15;
    return (float)(h >> 8) * (2.0f / 16777216.0f) - 1.0f;
}

// keys[r] = side bits of row r, vals[r] = r.  Shared memory: the hyperplanes
// (nb x dim) and their offsets.
__global__ void lsh_key_kernel(const float *x, int64_t n, int dim, int nb, int32_t *keys,
                               int32_t *vals) {
    extern __shared__ float H[];
    float *thr = H + nb * dim;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int e = threadIdx.x; e < nb * dim; e += blockDim.x) H[e] = plane_entry(e / dim, e % dim);
    __syncthreads();
    for (int j = warp; j < nb; j += nw) {
        // hyperplane j passes through data point ref_j
        const int64_t ref = (int64_t)((((uint64_t)(2 * j + 1) * 0x9E3779B97F4A7C15ull) >> 33) % (uint64_t)n);
        float acc = 0.f;
        for (int k = lane; k < dim; k += 32) acc = fmaf(H[j * dim + k], x[ref * dim + k], acc);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) thr[j] = acc;
    }
    __syncthreads();
    const int64_t gw = (int64_t)blockIdx.x * nw + warp, tw = (int64_t)gridDim.x * nw;
    for (int64_t r = gw; r < n; r += tw) {
        float part[kMaxPlanes];
#pragma unroll
        for (int j = 0; j < kMaxPlanes; ++j) part[j] = 0.f;
        for (int k = lane; k < dim; k += 32) {
            const float v = x[r * dim + k];
#pragma unroll
            for (int j = 0; j < kMaxPlanes; ++j)
                if (j < nb) part[j] = fmaf(v, H[j * dim + k], part[j]);
        }
        int32_t key = 0;
#pragma unroll
        for (int j = 0; j < kMaxPlanes; ++j) {
            float sv = part[j];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) sv += __shfl_xor_sync(0xffffffffu, sv, o);
            if (j < nb && sv > thr[j]) key |= 1 << j;
        }
        if (lane == 0) {
            keys[r] = key;
            vals[r] = (int32_t)r;
        }
    }
}

__global__ void rank_kernel(const int32_t *order, int64_t n, int32_t *rank) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        rank[order[i]] = (int32_t)i;
}

// keys[i] = rank of list[i] (pivots) or of its pivot (followers), vals[i] = list[i]
__global__ void list_keys_kernel(const int32_t *list, int64_t m, const int32_t *rank,
                                 const int32_t *pivot_of, int32_t *keys, int32_t *vals) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = list[i];
        keys[i] = rank[pivot_of ? pivot_of[v] : v];
        vals[i] = v;
    }
}

int grid_of(int64_t n) {
    int64_t g = (n + 255) / 256;
    if (g > 8192) g = 8192;
    return g < 1 ? 1 : (int)g;
}

}  // namespace

cudaError_t launch_locality_order(const float *x, int64_t n, int32_t dim, int32_t *keys,
                                  int32_t *vals, int64_t *offs, int32_t *cursor, void *scan_tmp,
                                  size_t scan_tmp_bytes, int32_t *order, int32_t *rank,
                                  cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    // about eight vertices per key at least, at most 2^12 keys; a single key below
    // 16 vertices (the counting-sort scratch holds as many keys as the largest
    // segment has vertices)
    int nb = 0;
    while (nb < kMaxPlanes && ((int64_t)8 << (nb + 1)) <= n) ++nb;
    const size_t smem = sizeof(float) * ((size_t)nb * dim + nb + 1);
    cudaError_t e = cudaFuncSetAttribute(lsh_key_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    int64_t g = (n + 7) / 8;
    if (g > 4 * 1024) g = 4 * 1024;
    lsh_key_kernel<<<(unsigned)g, 256, smem, st>>>(x, n, dim, nb, keys, vals);
    note_launches(1);
    e = launch_bucket(keys, vals, n, nullptr, (int64_t)1 << nb, 0, offs, cursor, order, scan_tmp,
                      scan_tmp_bytes, st);
    if (e != cudaSuccess) return e;
    rank_kernel<<<grid_of(n), 256, 0, st>>>(order, n, rank);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t order_search_lists(const int32_t *rank, const int32_t *pivot_of, int32_t *pivots,
                               int64_t np, int32_t *followers, int64_t nf, int64_t n,
                               int32_t *keys, int32_t *vals, int64_t *offs, int32_t *cursor,
                               void *scan_tmp, size_t scan_tmp_bytes, cudaStream_t st) {
    cudaError_t e = cudaSuccess;
    if (np > 0) {
        list_keys_kernel<<<grid_of(np), 256, 0, st>>>(pivots, np, rank, nullptr, keys, vals);
        note_launches(1);
        e = launch_bucket(keys, vals, np, nullptr, n, 0, offs, cursor, pivots, scan_tmp,
                          scan_tmp_bytes, st);
        if (e != cudaSuccess) return e;
    }
    if (nf > 0) {
        list_keys_kernel<<<grid_of(nf), 256, 0, st>>>(followers, nf, rank, pivot_of, keys, vals);
        note_launches(1);
        e = launch_bucket(keys, vals, nf, nullptr, n, 0, offs, cursor, followers, scan_tmp,
                          scan_tmp_bytes, st);
    }
    return e;
}

}  // namespace rnsm
