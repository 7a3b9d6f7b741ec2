// K3 and small helpers: counting sort of (key, value) pairs into CSR
// (histogram, exclusive scan, scatter), per-row sorts, the pairs of the
// reverse-kNN inversion, input validation, list initialisation and the
// medoid of a vector set.
//
// The scatter claims slots with atomics, so the order inside a row depends
// on scheduling; every consumer either sorts its rows (launch_sort_rows) or
// treats them as sets (the prune sorts its pool by (distance, id), pivot
// selection uses set sizes and membership), so results are deterministic.
#include <float.h>
#include <math.h>

#include <atomic>

#include "internal.h"

namespace rnsm {

namespace {
std::atomic<long long> g_launches{0};
}

void note_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
long long launches_so_far() { return g_launches.load(std::memory_order_relaxed); }

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;

__global__ void count_kernel(const int32_t *keys, int64_t cap, const unsigned long long *count,
                             int64_t nkeys, int32_t key_offset, int32_t *cnt) {
    const int64_t n = count ? (int64_t)min((unsigned long long)cap, *count) : cap;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = (int64_t)keys[i] - key_offset;
        if (k >= 0 && k < nkeys) atomicAdd(&cnt[k], 1);
    }
}

__device__ int64_t block_exclusive_scan(int64_t v, int64_t *warp_sums, int64_t &total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int64_t w = lane < (int)(blockDim.x >> 5) ? warp_sums[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < (int)(blockDim.x >> 5)) warp_sums[lane] = w;
    }
    __syncthreads();
    const int64_t before = warp == 0 ? 0 : warp_sums[warp - 1];
    total = warp_sums[(blockDim.x >> 5) - 1];
    __syncthreads();
    return before + x - v;
}

__global__ void __launch_bounds__(kScanThreads) tile_sum_kernel(const int32_t *cnt, int64_t n,
                                                                int64_t *tile_sums) {
    __shared__ int64_t ws[kScanThreads / 32];
    const int64_t t0 = (int64_t)blockIdx.x * kScanTile;
    int64_t s = 0;
    for (int j = 0; j < kScanItems; ++j) {
        const int64_t i = t0 + (int64_t)threadIdx.x * kScanItems + j;
        if (i < n) s += cnt[i];
    }
    int64_t total;
    block_exclusive_scan(s, ws, total);
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(1024) scan_tiles_kernel(int64_t *tile_sums, int64_t ntiles) {
    __shared__ int64_t ws[32];
    __shared__ int64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t b = 0; b < ntiles; b += blockDim.x) {
        const int64_t i = b + threadIdx.x;
        const int64_t v = i < ntiles ? tile_sums[i] : 0;
        int64_t total;
        const int64_t ex = block_exclusive_scan(v, ws, total);
        if (i < ntiles) tile_sums[i] = carry + ex;
        __syncthreads();
        if (threadIdx.x == 0) carry += total;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kScanThreads) scan_apply_kernel(const int32_t *cnt, int64_t n,
                                                                  const int64_t *tile_prefix,
                                                                  int64_t *offs) {
    __shared__ int64_t ws[kScanThreads / 32];
    const int64_t t0 = (int64_t)blockIdx.x * kScanTile;
    int64_t v[kScanItems];
    int64_t s = 0;
    for (int j = 0; j < kScanItems; ++j) {
        const int64_t i = t0 + (int64_t)threadIdx.x * kScanItems + j;
        v[j] = i < n ? cnt[i] : 0;
        s += v[j];
    }
    int64_t total;
    int64_t run = block_exclusive_scan(s, ws, total) + tile_prefix[blockIdx.x];
    for (int j = 0; j < kScanItems; ++j) {
        const int64_t i = t0 + (int64_t)threadIdx.x * kScanItems + j;
        if (i < n) offs[i] = run;
        run += v[j];
        if (i == n - 1) offs[n] = run;
    }
}

__global__ void scatter_kernel(const int32_t *keys, const int32_t *vals, int64_t cap,
                               const unsigned long long *count, int64_t nkeys, int32_t key_offset,
                               const int64_t *offs, int32_t *cursor, int32_t *out) {
    const int64_t n = count ? (int64_t)min((unsigned long long)cap, *count) : cap;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = (int64_t)keys[i] - key_offset;
        if (k >= 0 && k < nkeys) out[offs[k] + atomicAdd(&cursor[k], 1)] = vals[i];
    }
}

// One warp per row; rows up to 4096 entries sorted in shared memory.
constexpr int kRowSortCap = 4096;
constexpr int kRowSortWarps = 4;

__global__ void __launch_bounds__(kRowSortWarps * 32) sort_rows_kernel(const int64_t *offs,
                                                                       int32_t *ids, int64_t nrows,
                                                                       int32_t *err) {
    extern __shared__ int32_t sbuf[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int32_t *buf = sbuf + warp * kRowSortCap;
    for (int64_t r = (int64_t)blockIdx.x * kRowSortWarps + warp; r < nrows;
         r += (int64_t)gridDim.x * kRowSortWarps) {
        const int64_t lo = offs[r], n = offs[r + 1] - lo;
        if (n <= 1) continue;
        if (n > kRowSortCap) {
            if (lane == 0) atomicOr(err, 32);
            continue;
        }
        if (n <= 32) {
            int32_t v = lane < n ? ids[lo + lane] : INT32_MAX;
            float dummy = 0.f;
            warp_sort32(dummy, v);  // all keys share distance 0: orders by id
            if (lane < n) ids[lo + lane] = v;
            continue;
        }
        int np = 32;
        while (np < n) np <<= 1;
        for (int j = lane; j < np; j += 32) buf[j] = j < n ? ids[lo + j] : INT32_MAX;
        __syncwarp();
        for (int k = 2; k <= np; k <<= 1)
            for (int j = k >> 1; j > 0; j >>= 1) {
                for (int x = lane; x < np; x += 32) {
                    const int y = x ^ j;
                    if (y > x) {
                        const bool up = (x & k) == 0;
                        if ((buf[x] > buf[y]) == up) {
                            int32_t t = buf[x]; buf[x] = buf[y]; buf[y] = t;
                        }
                    }
                }
                __syncwarp();
            }
        for (int j = lane; j < n; j += 32) ids[lo + j] = buf[j];
        __syncwarp();
    }
}

__global__ void rk_pairs_kernel(const int32_t *nplus, int64_t n, int32_t k_plus, int32_t k,
                                int32_t *keys, int32_t *vals, unsigned long long *count) {
    const int64_t total = n * k;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t y = e / k;
        const int j = (int)(e - y * k);
        keys[e] = nplus[y * k_plus + j];
        vals[e] = (int32_t)y;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *count = (unsigned long long)total;
}

__global__ void validate_ids_kernel(const int32_t *ids, int64_t total, int64_t bound, int32_t lo,
                                    int32_t *err) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = ids[i];
        if (v < lo || v >= bound) atomicOr(err, 1);
    }
}

__global__ void validate_vecs_kernel(const float *v, int64_t count, int32_t *err) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (!isfinite(v[i])) atomicOr(err, 2);
    }
}

__global__ void init_lists_kernel(const int32_t *adj, int64_t n, int32_t r_in, int32_t offset,
                                  int32_t *out, int32_t R) {
    const int64_t total = n * R;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = e / R;
        const int j = (int)(e - v * R);
        int32_t u = j < r_in ? adj[v * r_in + j] : -1;
        out[e] = u >= 0 ? u + offset : -1;
    }
}

__global__ void fill_kernel(int32_t *p, int64_t count, int32_t value) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x)
        p[i] = value;
}

// Medoid, FP64, deterministic: fixed block partition, fixed summation order.
constexpr int kMedBlocks = 512;

__global__ void medoid_colsum_kernel(const float *v, int64_t n, int32_t dim, double *part) {
    const int64_t per = (n + gridDim.x - 1) / gridDim.x;
    const int64_t r0 = blockIdx.x * per, r1 = min(n, r0 + per);
    for (int j = threadIdx.x; j < dim; j += blockDim.x) {
        double s = 0.0;
        for (int64_t r = r0; r < r1; ++r) s += (double)v[r * dim + j];
        part[(int64_t)blockIdx.x * dim + j] = s;
    }
}

__global__ void medoid_centroid_kernel(const double *part, int nblk, int64_t n, int32_t dim,
                                       double *c) {
    for (int j = threadIdx.x; j < dim; j += blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < nblk; ++b) s += part[(int64_t)b * dim + j];
        c[j] = s / (double)n;
    }
}

__global__ void medoid_argmin_kernel(const float *v, int64_t n, int32_t dim, int32_t metric,
                                     const double *c, double *bd, int32_t *bi) {
    __shared__ double sd[32];
    __shared__ int32_t si[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int64_t per = (n + gridDim.x - 1) / gridDim.x;
    const int64_t r0 = blockIdx.x * per, r1 = min(n, r0 + per);
    double best = INFINITY;
    int32_t bid = INT32_MAX;
    for (int64_t r = r0 + warp; r < r1; r += nw) {
        double s = 0.0;
        for (int j = lane; j < dim; j += 32) {
            const double x = (double)v[r * dim + j];
            if (metric == 0) {
                const double t = x - c[j];
                s += t * t;
            } else {
                s += x * c[j];
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (metric != 0) s = 1.0 - s;
        if (s < best || (s == best && r < bid)) { best = s; bid = (int32_t)r; }
    }
    if (lane == 0) { sd[warp] = best; si[warp] = bid; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < nw; ++w)
            if (sd[w] < best || (sd[w] == best && si[w] < bid)) { best = sd[w]; bid = si[w]; }
        bd[blockIdx.x] = best;
        bi[blockIdx.x] = bid;
    }
}

__global__ void medoid_final_kernel(const double *bd, const int32_t *bi, int nblk, int32_t *out) {
    double best = INFINITY;
    int32_t bid = INT32_MAX;
    for (int b = 0; b < nblk; ++b)
        if (bd[b] < best || (bd[b] == best && bi[b] < bid)) { best = bd[b]; bid = bi[b]; }
    *out = bid;
}

__global__ void max_row_kernel(const int64_t *offs, int64_t n, int32_t *out) {
    int32_t m = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        m = max(m, (int32_t)(offs[i + 1] - offs[i]));
    atomicMax(out, m);
}

int grid_for(int64_t work, int threads) {
    int64_t g = (work + threads - 1) / threads;
    if (g > 4096) g = 4096;
    if (g < 1) g = 1;
    return (int)g;
}

}  // namespace

size_t bucket_scan_tmp_bytes(int64_t nkeys) {
    return (size_t)((nkeys + kScanTile - 1) / kScanTile + 1) * sizeof(int64_t);
}

cudaError_t launch_bucket(const int32_t *keys, const int32_t *vals, int64_t cap,
                          const unsigned long long *count, int64_t nkeys, int32_t key_offset,
                          int64_t *offs, int32_t *cursor, int32_t *out_vals, void *scan_tmp,
                          size_t scan_tmp_bytes, cudaStream_t st) {
    if (scan_tmp_bytes < bucket_scan_tmp_bytes(nkeys)) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(cursor, 0, sizeof(int32_t) * (size_t)nkeys, st);
    if (e != cudaSuccess) return e;
    if (cap > 0) {
        count_kernel<<<grid_for(cap, 256), 256, 0, st>>>(keys, cap, count, nkeys, key_offset,
                                                         cursor);
        note_launches(2);  // count + scatter
    }
    const int64_t ntiles = (nkeys + kScanTile - 1) / kScanTile;
    int64_t *tiles = static_cast<int64_t *>(scan_tmp);
    if (ntiles > 0) {
        tile_sum_kernel<<<(unsigned)ntiles, kScanThreads, 0, st>>>(cursor, nkeys, tiles);
        scan_tiles_kernel<<<1, 1024, 0, st>>>(tiles, ntiles);
        scan_apply_kernel<<<(unsigned)ntiles, kScanThreads, 0, st>>>(cursor, nkeys, tiles, offs);
        note_launches(3);
    } else {
        e = cudaMemsetAsync(offs, 0, sizeof(int64_t), st);
        if (e != cudaSuccess) return e;
    }
    e = cudaMemsetAsync(cursor, 0, sizeof(int32_t) * (size_t)nkeys, st);
    if (e != cudaSuccess) return e;
    if (cap > 0)
        scatter_kernel<<<grid_for(cap, 256), 256, 0, st>>>(keys, vals, cap, count, nkeys, key_offset,
                                                           offs, cursor, out_vals);
    return cudaGetLastError();
}

cudaError_t launch_sort_rows(const int64_t *offs, int32_t *ids, int64_t nrows, int32_t *err,
                             cudaStream_t st) {
    if (nrows <= 0) return cudaSuccess;
    const size_t smem = (size_t)kRowSortWarps * kRowSortCap * sizeof(int32_t);
    cudaError_t e = cudaFuncSetAttribute(sort_rows_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int64_t g = (nrows + kRowSortWarps - 1) / kRowSortWarps;
    if (g > 8192) g = 8192;
    sort_rows_kernel<<<(unsigned)g, kRowSortWarps * 32, smem, st>>>(offs, ids, nrows, err);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_rk_pairs(const int32_t *nplus, int64_t n, int32_t k_plus, int32_t k,
                            int32_t *keys, int32_t *vals, unsigned long long *count,
                            cudaStream_t st) {
    rk_pairs_kernel<<<grid_for(n * k, 256), 256, 0, st>>>(nplus, n, k_plus, k, keys, vals, count);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_validate_graph(const int32_t *adj, int64_t n, int32_t r_in, int32_t *err,
                                  cudaStream_t st) {
    return launch_validate_ids(adj, n * r_in, n, 1, err, st);
}

cudaError_t launch_validate_ids(const int32_t *ids, int64_t count, int64_t bound,
                                int32_t allow_minus1, int32_t *err, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    validate_ids_kernel<<<grid_for(count, 256), 256, 0, st>>>(ids, count, bound,
                                                              allow_minus1 ? -1 : 0, err);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_validate_vecs(const float *v, int64_t count, int32_t *err, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    validate_vecs_kernel<<<grid_for(count, 256), 256, 0, st>>>(v, count, err);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_init_lists(const int32_t *adj, int64_t n, int32_t r_in, int32_t offset,
                              int32_t *out, int32_t R, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    init_lists_kernel<<<grid_for(n * R, 256), 256, 0, st>>>(adj, n, r_in, offset, out, R);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_fill(int32_t *p, int64_t count, int32_t value, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    fill_kernel<<<grid_for(count, 256), 256, 0, st>>>(p, count, value);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_max_row(const int64_t *offs, int64_t n, int32_t *out, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(int32_t), st);
    if (e != cudaSuccess || n <= 0) return e;
    max_row_kernel<<<grid_for(n, 256), 256, 0, st>>>(offs, n, out);
    note_launches(1);
    return cudaGetLastError();
}

size_t medoid_tmp_bytes(int64_t n, int32_t dim) {
    (void)n;
    return (size_t)kMedBlocks * dim * sizeof(double) + dim * sizeof(double) +
           kMedBlocks * (sizeof(double) + sizeof(int32_t)) + 64;
}

cudaError_t launch_medoid(const float *v, int64_t n, int32_t dim, int32_t metric, double *tmp,
                          size_t tmp_bytes, int32_t *out, cudaStream_t st) {
    if (tmp_bytes < medoid_tmp_bytes(n, dim) || n < 1) return cudaErrorInvalidValue;
    double *part = tmp;
    double *c = part + (size_t)kMedBlocks * dim;
    double *bd = c + dim;
    int32_t *bi = reinterpret_cast<int32_t *>(bd + kMedBlocks);
    medoid_colsum_kernel<<<kMedBlocks, 128, 0, st>>>(v, n, dim, part);
    medoid_centroid_kernel<<<1, 256, 0, st>>>(part, kMedBlocks, n, dim, c);
    medoid_argmin_kernel<<<kMedBlocks, 256, 0, st>>>(v, n, dim, metric, c, bd, bi);
    medoid_final_kernel<<<1, 1, 0, st>>>(bd, bi, kMedBlocks, out);
    note_launches(4);
    return cudaGetLastError();
}

}  // namespace rnsm
