// S3 on the device: the lazy-greedy pivot selection of Algorithm 2 (Phase 2)
// computed in parallel rounds with the same result.
//
// The lazy greedy (max-heap on (gain, lower id), stale entries reinserted)
// selects, at every step, the uncovered vertex of largest key
// (|R_k(x) \ Covered|, -x).  Selecting y can change x's key or cover x only if
// y is in x's conflict set
//     Conf(x) = N_k(x) u R_k(x) u { N_k(z) : z in R_k(x), z uncovered }
// (y covers x iff x in R_k(y) iff y in N_k(x); y lowers x's gain iff y covers
// an uncovered z in R_k(x), i.e. y = z or y in N_k(z)), and the relation is
// symmetric.  A vertex whose key beats every uncovered member of its conflict
// set keeps its key until the sequential greedy reaches it, so the sequential
// greedy selects it with the same follower set F_x = R_k(x) \ Covered; such
// local maxima never conflict with each other, so one round selects all of
// them at once.  The global maximum is always a local maximum, so every round
// makes progress.
#include "internal.h"

namespace rnsm {

namespace {

__global__ void piv_init_kernel(int64_t n, uint8_t *covered, int32_t *pivot_of) {
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < n;
         x += (int64_t)gridDim.x * blockDim.x) {
        covered[x] = 0;
        pivot_of[x] = -2;
    }
}

// key = (gain << 32) | (~x): larger gain first, then the lower id; 0 if covered.
__global__ void piv_gain_kernel(int64_t n, const int64_t *offs, const int32_t *ids,
                                const uint8_t *covered, unsigned long long *key) {
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < n;
         x += (int64_t)gridDim.x * blockDim.x) {
        if (covered[x]) {
            key[x] = 0ull;
            continue;
        }
        unsigned long long g = 0;
        for (int64_t e = offs[x]; e < offs[x + 1]; ++e) g += covered[ids[e]] ? 0 : 1;
        key[x] = (g << 32) | (unsigned long long)(0xffffffffu - (uint32_t)x);
    }
}

__global__ void piv_select_kernel(int64_t n, const int32_t *nplus, int32_t k_plus, int32_t k,
                                  const int64_t *offs, const int32_t *ids, const uint8_t *covered,
                                  const unsigned long long *key, uint8_t *sel) {
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < n;
         x += (int64_t)gridDim.x * blockDim.x) {
        if (covered[x]) {
            sel[x] = 0;
            continue;
        }
        const unsigned long long kx = key[x];
        bool ok = true;
        const int32_t *nx = nplus + x * k_plus;
        for (int j = 0; ok && j < k; ++j) {
            const int32_t y = nx[j];
            if (y >= 0 && key[y] > kx) ok = false;
        }
        for (int64_t e = offs[x]; ok && e < offs[x + 1]; ++e) {
            const int32_t z = ids[e];
            if (key[z] > kx) { ok = false; break; }
            if (covered[z]) continue;
            const int32_t *nz = nplus + (int64_t)z * k_plus;
            for (int j = 0; j < k; ++j) {
                const int32_t y = nz[j];
                if (y >= 0 && y != (int32_t)x && key[y] > kx) { ok = false; break; }
            }
        }
        sel[x] = ok ? 1 : 0;
    }
}

__global__ void piv_apply_kernel(int64_t n, const int64_t *offs, const int32_t *ids,
                                 const uint8_t *sel, uint8_t *covered, int32_t *pivot_of,
                                 unsigned long long *newly) {
    unsigned long long cnt = 0;
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < n;
         x += (int64_t)gridDim.x * blockDim.x) {
        if (!sel[x]) continue;
        // selected vertices never share an uncovered reverse neighbour
        for (int64_t e = offs[x]; e < offs[x + 1]; ++e) {
            const int32_t y = ids[e];
            if (!covered[y]) {
                covered[y] = 1;
                pivot_of[y] = (int32_t)x;
                ++cnt;
            }
        }
        covered[x] = 1;
        pivot_of[x] = -1;
        ++cnt;
    }
    if (cnt) atomicAdd(newly, cnt);
}

__global__ void piv_compact_kernel(int64_t n, const int32_t *pivot_of, int32_t *pivots,
                                   int32_t *followers, unsigned long long *counts) {
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < n;
         x += (int64_t)gridDim.x * blockDim.x) {
        if (pivot_of[x] == -1) pivots[atomicAdd(&counts[0], 1ull)] = (int32_t)x;
        else followers[atomicAdd(&counts[1], 1ull)] = (int32_t)x;
    }
}

int grid_n(int64_t n) {
    int64_t g = (n + 255) / 256;
    if (g > 8192) g = 8192;
    return g < 1 ? 1 : (int)g;
}

}  // namespace

size_t pivot_tmp_bytes(int64_t n) {
    return (size_t)n * (sizeof(unsigned long long) + 2) + 256;
}

cudaError_t select_pivots_device(const int32_t *nplus, int64_t n, int32_t k_plus, int32_t k,
                                 const int64_t *offs, const int32_t *ids, int32_t *pivot_of,
                                 int32_t *pivots, int32_t *followers, int64_t *n_pivots,
                                 int64_t *n_followers, int32_t *rounds, void *tmp,
                                 unsigned long long *counters, cudaStream_t st) {
    if (n <= 0) {
        *n_pivots = *n_followers = 0;
        return cudaSuccess;
    }
    unsigned long long *key = static_cast<unsigned long long *>(tmp);
    uint8_t *covered = reinterpret_cast<uint8_t *>(key + n);
    uint8_t *sel = covered + n;
    const int g = grid_n(n);
    piv_init_kernel<<<g, 256, 0, st>>>(n, covered, pivot_of);
    note_launches(1);
    int64_t done = 0;
    int r = 0;
    // Rounds in batches: extra rounds after convergence select nothing.
    constexpr int kBatch = 4;
    while (done < n) {
        cudaError_t e = cudaMemsetAsync(counters, 0, sizeof(unsigned long long), st);
        if (e != cudaSuccess) return e;
        for (int b = 0; b < kBatch; ++b) {
            piv_gain_kernel<<<g, 256, 0, st>>>(n, offs, ids, covered, key);
            piv_select_kernel<<<g, 256, 0, st>>>(n, nplus, k_plus, k, offs, ids, covered, key, sel);
            piv_apply_kernel<<<g, 256, 0, st>>>(n, offs, ids, sel, covered, pivot_of, counters);
            note_launches(3);
        }
        r += kBatch;
        unsigned long long newly = 0;
        e = cudaMemcpyAsync(&newly, counters, sizeof(newly), cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) return e;
        e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return e;
        if (newly == 0) return cudaErrorUnknown;  // cannot happen: a round always selects
        done += (int64_t)newly;
    }
    cudaError_t e = cudaMemsetAsync(counters, 0, 2 * sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    piv_compact_kernel<<<g, 256, 0, st>>>(n, pivot_of, pivots, followers, counters);
    note_launches(1);
    unsigned long long c[2] = {0, 0};
    e = cudaMemcpyAsync(c, counters, sizeof(c), cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return e;
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    *n_pivots = (int64_t)c[0];
    *n_followers = (int64_t)c[1];
    if (rounds) *rounds = r;
    return cudaGetLastError();
}

}  // namespace rnsm
