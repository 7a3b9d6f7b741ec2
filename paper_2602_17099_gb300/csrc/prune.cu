// K2: occlusion prune of UpdateGraph (Section 4.2; the RNG-variant edge
// selection of Section 2.2), one CTA per owner vertex, persistent.
//
// For owner v with pool W: gather and deduplicate W (drop v and -1),
// compute d(v, c) for every candidate, sort by (d, id), then walk the order
// in tile passes.  A pass stages the rows of the candidates kept so far plus
// the next chunk of up to 64 candidates in shared memory, builds the
// candidate-by-candidate distance tile for every pair (earlier, chunk) with
// FP32 direct differences (register-blocked 4x4 per thread), and one warp
// scans the chunk in order: candidate c is occluded iff some kept s has
// fmaf(alpha, d(s,c), -d(v,c)) <= 0 (one rounding, so the sign is that of
// the exact alpha*d(s,c) - d(v,c)), decided with warp ballots.  The walk stops
// once R candidates are kept.
#include <float.h>

#include "internal.h"

namespace rnsm {

namespace {

constexpr int kThreads = 128;
constexpr int kTile = 64;       // candidates per pass
constexpr int kDch = 128;       // dimensions staged per sub-pass
constexpr int kStride = kDch + 4;  // staged row stride (floats): 33 float4, odd => no bank conflicts
constexpr int kNB = 4;          // 4x4 pair blocks per thread (rows <= 128, chunk <= 64)
constexpr int kPoolCapMax = 4096;  // larger pools set error bit 16

struct Smem {
    float *rows;          // rows_cap * kStride
    const float **rptr;   // rows_cap
    float *tile;          // rows_cap * kTile
    float *pd;            // pool_cap
    int32_t *pid;         // pool_cap
    int32_t *tmp;         // pool_cap
    int32_t *krow;        // R
    int32_t *kid;         // R
};

size_t smem_bytes(int rows_cap, int pool_cap, int R) {
    return (size_t)rows_cap * kStride * 4 + (size_t)rows_cap * sizeof(void *) +
           (size_t)rows_cap * kTile * 4 + (size_t)pool_cap * 12 + (size_t)R * 8 + 64;
}

__device__ __forceinline__ void carve(unsigned char *p, int rows_cap, int pool_cap, int R, Smem &s) {
    s.rows = reinterpret_cast<float *>(p);
    s.rptr = reinterpret_cast<const float **>(s.rows + (size_t)rows_cap * kStride);
    s.tile = reinterpret_cast<float *>(s.rptr + rows_cap);
    s.pd = s.tile + (size_t)rows_cap * kTile;
    s.pid = reinterpret_cast<int32_t *>(s.pd + pool_cap);
    s.tmp = s.pid + pool_cap;
    s.krow = s.tmp + pool_cap;
    s.kid = s.krow + R;
}

__global__ void __launch_bounds__(kThreads) prune_kernel(const PruneArgs a, int rows_cap,
                                                         int pool_cap, int chunk) {
    extern __shared__ __align__(16) unsigned char smem[];
    Smem s;
    carve(smem, rows_cap, pool_cap, a.R, s);
    __shared__ int64_t sh_i;  // first owner of the claimed chunk
    __shared__ int sh_np, sh_nk, sh_ebase;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int dim = a.dim, F4 = dim >> 2;
    const int R = a.R;

    for (;;) {
        if (tid == 0) sh_i = atomicAdd(a.work, chunk);
        __syncthreads();
        const int64_t i0 = sh_i;
        if (i0 >= a.n_owners) break;
        const int64_t i1 = min(a.n_owners, i0 + chunk);
      for (int64_t i = i0; i < i1; ++i) {
        const int32_t owner = a.owner_ids ? a.owner_ids[i] : (int32_t)(a.owner_base + i);
        int64_t c_lo = 0, c_hi = 0;
        if (a.csr_offs) {
            c_lo = a.csr_offs[i];
            c_hi = a.csr_offs[i + 1];
        }
        if (a.skip_empty_csr && c_hi == c_lo) {
            __syncthreads();
            continue;
        }
        const int64_t np_raw = (int64_t)a.lenA + a.lenB + (c_hi - c_lo);
        if (np_raw > pool_cap) {
            if (tid == 0) atomicOr(a.err, 16);
            __syncthreads();
            continue;
        }

        // 1. Gather the pool.
        for (int j = tid; j < np_raw; j += kThreads) {
            int32_t id;
            if (j < a.lenA) {
                id = a.listA[(int64_t)owner * a.lenA + j];
            } else if (j < a.lenA + a.lenB) {
                id = a.listB[i * a.strideB + (j - a.lenA)];
                if (id >= 0) id += a.offB;
            } else {
                id = a.csr_ids[c_lo + (j - a.lenA - a.lenB)];
            }
            s.pid[j] = id;
        }
        if (tid == 0) sh_np = 0;
        __syncthreads();
        // 2. Drop -1, the owner and duplicates (first occurrence survives).
        for (int j = tid; j < np_raw; j += kThreads) {
            const int32_t id = s.pid[j];
            bool ok = id >= 0 && id != owner;
            for (int t = 0; ok && t < j; ++t)
                if (s.pid[t] == id) ok = false;
            if (ok) s.tmp[atomicAdd(&sh_np, 1)] = id;
        }
        __syncthreads();
        const int np = sh_np;
        for (int j = tid; j < np; j += kThreads) s.pid[j] = s.tmp[j];
        __syncthreads();

        // 3. d(v, c) for every candidate: one warp per candidate, 4 at a time.
        {
            const float *orow = seg_row(a.segs, owner, dim);
            for (int c0 = warp * 4; c0 < np; c0 += 16) {
                const float *rw[4];
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    rw[u] = c0 + u < np ? seg_row(a.segs, s.pid[c0 + u], dim) : orow;
                float v[4] = {0.f, 0.f, 0.f, 0.f};
                for (int f = lane; f < F4; f += 32) {
                    const float4 o = ldg4(orow + 4 * f);
                    float4 x[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) x[u] = ldg4(rw[u] + 4 * f);
                    if (a.metric == 0) {
#pragma unroll
                        for (int u = 0; u < 4; ++u) v[u] = l2_acc(v[u], o, x[u]);
                    } else {
#pragma unroll
                        for (int u = 0; u < 4; ++u) v[u] = ip_acc(v[u], o, x[u]);
                    }
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
#pragma unroll
                    for (int off = 16; off > 0; off >>= 1)
                        v[u] += __shfl_xor_sync(0xffffffffu, v[u], off);
                }
                if (lane == 0) {
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        if (c0 + u < np) s.pd[c0 + u] = a.metric == 0 ? v[u] : 1.0f - v[u];
                }
            }
        }
        // 4. Sort (pd, pid) by (distance, id): bitonic over the next power of two.
        int npad = 1;
        while (npad < np) npad <<= 1;
        for (int j = np + tid; j < npad; j += kThreads) {
            s.pd[j] = INFINITY;
            s.pid[j] = INT32_MAX;
        }
        __syncthreads();
        for (int k = 2; k <= npad; k <<= 1) {
            for (int j = k >> 1; j > 0; j >>= 1) {
                for (int x = tid; x < npad; x += kThreads) {
                    const int y = x ^ j;
                    if (y > x) {
                        const bool up = (x & k) == 0;
                        const bool gt = lex_less(s.pd[y], s.pid[y], s.pd[x], s.pid[x]);
                        if (gt == up) {
                            float td = s.pd[x]; s.pd[x] = s.pd[y]; s.pd[y] = td;
                            int32_t ti = s.pid[x]; s.pid[x] = s.pid[y]; s.pid[y] = ti;
                        }
                    }
                }
                __syncthreads();
            }
        }

        // 5. Walk in order.
        int nk = 0;
        if (a.keep_all_if_fit && np <= R) {
            for (int j = tid; j < np; j += kThreads) s.kid[j] = s.pid[j];
            nk = np;
        } else {
            int pos = 0;
            while (pos < np && nk < R) {
                const int cs = min(kTile, np - pos);
                const int nrows = nk + cs;
                const int nA = (nrows + 3) >> 2, nB = (cs + 3) >> 2;
                const int nblk = nA * nB;
                // staged rows: kept [0, nk), chunk [nk, nrows)
                for (int r = tid; r < nrows; r += kThreads) {
                    const int32_t id = r < nk ? s.kid[r] : s.pid[pos + r - nk];
                    s.rptr[r] = seg_row(a.segs, id, dim);
                }
                for (int r = nrows + tid; r < 4 * nA; r += kThreads)
                    s.rptr[r] = seg_row(a.segs, owner, dim);  // padding rows: any valid row
                for (int j = tid; j < nk; j += kThreads) s.krow[j] = j;
                __syncthreads();
                float acc[kNB][4][4];
#pragma unroll
                for (int t = 0; t < kNB; ++t)
#pragma unroll
                    for (int p = 0; p < 4; ++p)
#pragma unroll
                        for (int q = 0; q < 4; ++q) acc[t][p][q] = 0.f;
                for (int d0 = 0; d0 < dim; d0 += kDch) {
                    const int dc4 = min(kDch, dim - d0) >> 2;
                    const int rows4 = 4 * nA;
                    for (int e = tid; e < rows4 * dc4; e += kThreads) {
                        const int r = e / dc4, f = e - r * dc4;
                        const float4 v = ldg4(s.rptr[r] + d0 + 4 * f);
                        *reinterpret_cast<float4 *>(s.rows + (size_t)r * kStride + 4 * f) = v;
                    }
                    __syncthreads();
#pragma unroll
                    for (int t = 0; t < kNB; ++t) {
                        const int b = tid + kThreads * t;
                        if (b < nblk) {
                            const int ba = b / nB, bb = b - ba * nB;
                            const float *ra[4], *rb[4];
#pragma unroll
                            for (int p = 0; p < 4; ++p) {
                                ra[p] = s.rows + (size_t)(ba + nA * p) * kStride;
                                int rbi = nk + bb + nB * p;
                                if (rbi >= 4 * nA) rbi = 0;
                                rb[p] = s.rows + (size_t)rbi * kStride;
                            }
                            for (int f = 0; f < dc4; ++f) {
                                float4 xa[4], xb[4];
#pragma unroll
                                for (int p = 0; p < 4; ++p) {
                                    xa[p] = *reinterpret_cast<const float4 *>(ra[p] + 4 * f);
                                    xb[p] = *reinterpret_cast<const float4 *>(rb[p] + 4 * f);
                                }
                                if (a.metric == 0) {
#pragma unroll
                                    for (int p = 0; p < 4; ++p)
#pragma unroll
                                        for (int q = 0; q < 4; ++q)
                                            acc[t][p][q] = l2_acc(acc[t][p][q], xa[p], xb[q]);
                                } else {
#pragma unroll
                                    for (int p = 0; p < 4; ++p)
#pragma unroll
                                        for (int q = 0; q < 4; ++q)
                                            acc[t][p][q] = ip_acc(acc[t][p][q], xa[p], xb[q]);
                                }
                            }
                        }
                    }
                    __syncthreads();
                }
#pragma unroll
                for (int t = 0; t < kNB; ++t) {
                    const int b = tid + kThreads * t;
                    if (b < nblk) {
                        const int ba = b / nB, bb = b - ba * nB;
#pragma unroll
                        for (int p = 0; p < 4; ++p)
#pragma unroll
                            for (int q = 0; q < 4; ++q) {
                                const int ar = ba + nA * p, bc = bb + nB * q;
                                if (ar < nrows && bc < cs && ar < nk + bc)
                                    s.tile[ar * kTile + bc] =
                                        a.metric == 0 ? acc[t][p][q] : 1.0f - acc[t][p][q];
                            }
                    }
                }
                __syncthreads();
                if (warp == 0) {
                    int nkk = nk;
                    for (int bc = 0; bc < cs && nkk < R; ++bc) {
                        const float dvc = s.pd[pos + bc];
                        bool occ = false;
                        for (int j0 = 0; j0 < nkk && !occ; j0 += 32) {
                            const int j = j0 + lane;
                            bool t = false;
                            if (j < nkk) t = fmaf(a.alpha, s.tile[s.krow[j] * kTile + bc], -dvc) <= 0.f;
                            occ = __any_sync(0xffffffffu, t);
                        }
                        if (!occ) {
                            if (lane == 0) {
                                s.krow[nkk] = nk + bc;
                                s.kid[nkk] = s.pid[pos + bc];
                            }
                            ++nkk;
                            __syncwarp();
                        }
                    }
                    if (lane == 0) sh_nk = nkk;
                }
                __syncthreads();
                nk = sh_nk;
                pos += cs;
            }
        }
        __syncthreads();

        // 6. Output and reverse-edge emission.
        int32_t *orow = a.out + (a.out_by_index ? i : (int64_t)owner) * R;
        for (int j = tid; j < R; j += kThreads) orow[j] = j < nk ? s.kid[j] : -1;
        if (a.eu && warp == 0) {
            int cnt = 0;
            for (int j0 = 0; j0 < nk; j0 += 32) {
                const int j = j0 + lane;
                const bool e = j < nk && s.kid[j] >= a.emit_lo && s.kid[j] < a.emit_hi;
                cnt += __popc(__ballot_sync(0xffffffffu, e));
            }
            if (lane == 0) sh_ebase = cnt ? (int)atomicAdd(a.ecount, (unsigned long long)cnt) : 0;
            __syncwarp();
            const int base = sh_ebase;
            int done = 0;
            for (int j0 = 0; j0 < nk; j0 += 32) {
                const int j = j0 + lane;
                const bool e = j < nk && s.kid[j] >= a.emit_lo && s.kid[j] < a.emit_hi;
                const unsigned m = __ballot_sync(0xffffffffu, e);
                if (e) {
                    const int slot = base + done + __popc(m & lanemask_lt());
                    a.eu[slot] = s.kid[j];
                    a.ev[slot] = owner;
                }
                done += __popc(m);
            }
        }
        __syncthreads();
      }
    }
}

}  // namespace

cudaError_t launch_prune(const PruneArgs &a, cudaStream_t st) {
    if (a.n_owners <= 0) return cudaSuccess;
    if (a.R > 64 || a.dim > 1024 || (a.dim & 3)) return cudaErrorInvalidValue;
    const int64_t maxpool = (int64_t)a.lenA + a.lenB + (a.csr_offs ? a.csr_max : 0);
    int pool_cap = 64;
    while (pool_cap < maxpool && pool_cap < kPoolCapMax) pool_cap <<= 1;
    const int rows_cap = ((a.R + kTile + 3) / 4) * 4;
    const size_t smem = smem_bytes(rows_cap, pool_cap, a.R);
    cudaError_t e = cudaFuncSetAttribute(prune_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, prune_kernel, kThreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    int64_t grid = (int64_t)sms * per_sm;
    // Sparse passes (most owners without CSR entries) claim owners 32 at a time.
    const int chunk = a.skip_empty_csr ? 32 : 1;
    int64_t want = (a.n_owners + chunk - 1) / chunk;
    if (want < grid) grid = want;
    prune_kernel<<<(unsigned)grid, kThreads, smem, st>>>(a, rows_cap, pool_cap, chunk);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace rnsm
