// K2: occlusion prune of UpdateGraph (Section 4.2; the RNG-variant edge
// selection of Section 2.2), one CTA per owner vertex, persistent.
//
// For owner v with pool W: gather and deduplicate W (drop v and -1), order
// the candidates by (d(v,c), id) and walk them: c is kept unless a kept s has
// fmaf(alpha, d(s,c), -d(v,c)) <= 0 (one rounding, so the sign is that of the
// exact alpha*d(s,c) - d(v,c)); the walk stops once R are kept.
//
// Every FP32 distance here is the same fixed chain, acc = fmaf(a_i - b_i,
// a_i - b_i, acc) (or fmaf(a_i, b_i, acc), d = 1 - acc, for inner product)
// over i = 0 .. dim-1 in order, whichever code path computes it.
//
// Fast path (pool <= kFastMax): the owner row and all candidate rows are
// staged once in shared memory and one register-blocked pass builds the
// owner distances and the whole candidate-by-candidate triangle; the
// triangle then replaces the staged rows in the same buffer.  Slow path
// (larger pools): owner distances first, then passes that stage the kept rows
// plus the next 64 candidates.
#include <float.h>
#include <stdlib.h>

#include <map>
#include <mutex>

#include "internal.h"

namespace rnsm {

namespace {

constexpr int kThreads = 256;
constexpr int kDch = 128;           // dimensions staged per sub-pass
constexpr int kFastMax = 151;       // candidates of the one-tile path (rows = 1 + np <= 152)
constexpr int kNBFMax = 3;          // 4x4 pair blocks per thread, fast path (152 rows)
constexpr int kRowsNB1 = 88;        // rows whose triangle fits one block per thread
constexpr int kTile = 64;           // candidates per slow-path pass
constexpr int kNBS = 2;             // 4x4 pair blocks per thread, slow path
constexpr int kPoolCapMax = 4096;   // larger pools set error bit 16

// Staged row r starts at float4 index r*33 + (r >> 2): an odd stride plus a
// one-float4 shift every 4 rows, so 8 threads reading the same column of
// rows 4b+q (b = 0..7) hit 8 different bank groups.
__device__ __forceinline__ int srow4(int r) { return r * (kDch / 4 + 1) + (r >> 2); }
__host__ __device__ constexpr int rows_float4(int rows) { return rows * (kDch / 4 + 1) + rows / 4 + 1; }

// Upper-triangle index of the pair (a, b), a < b, among n rows.
__device__ __forceinline__ int tri(int a, int b, int n) { return a * (2 * n - a - 1) / 2 + (b - a - 1); }

struct Smem {
    float4 *rows;          // staged rows; reused for the triangle
    const float **rptr;    // row pointer of each staged row
    float *pd;             // pool_cap: d(v, c)
    int32_t *pid;          // pool_cap: candidate ids
    int32_t *prow;         // pool_cap: staged row of each candidate (fast path)
    int32_t *tmp;          // pool_cap
    int32_t *krow;         // R: staged row of each kept candidate
    int32_t *kid;          // R: kept ids in order
    float *stile;          // slow path: rows_cap * kTile pair distances
};

size_t smem_bytes(int rows_cap, int pool_cap, int R, bool slow) {
    size_t b = (size_t)rows_float4(rows_cap) * 16 + (size_t)rows_cap * sizeof(void *) +
               (size_t)pool_cap * 16 + (size_t)R * 8 + 64;
    if (slow) b += (size_t)rows_cap * kTile * 4;
    return b;
}

__device__ __forceinline__ void carve(unsigned char *p, int rows_cap, int pool_cap, int R,
                                      bool slow, Smem &s) {
    s.rows = reinterpret_cast<float4 *>(p);
    s.rptr = reinterpret_cast<const float **>(s.rows + rows_float4(rows_cap));
    s.pd = reinterpret_cast<float *>(s.rptr + rows_cap);
    s.pid = reinterpret_cast<int32_t *>(s.pd + pool_cap);
    s.prow = s.pid + pool_cap;
    s.tmp = s.prow + pool_cap;
    s.krow = s.tmp + pool_cap;
    s.kid = s.krow + R;
    s.stile = slow ? reinterpret_cast<float *>(s.kid + R) : nullptr;
}



// Stages float4 columns [d0/4, d0/4 + dc4) of rows [0, nrows4) (rptr) into
// smem; U loads per thread are issued before their stores so they overlap.
template <int NT, int U = 8>
__device__ __forceinline__ void stage_rows(float4 *rows, const float *const *rptr, int nrows4,
                                           int d0, int dc4) {
    // a warp per row, a lane per float4: coalesced 512-byte row reads, conflict-free
    // stores, U rows in flight per warp, no index division
    constexpr int NW = NT / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int f = lane; f - lane < dc4; f += 32) {
        const bool fin = f < dc4;
        for (int r0 = warp; r0 < nrows4; r0 += U * NW) {
            float4 v[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int r = r0 + u * NW;
                if (fin && r < nrows4) v[u] = ldg4(rptr[r] + d0 + 4 * f);
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int r = r0 + u * NW;
                if (fin && r < nrows4) rows[srow4(r) + f] = v[u];
            }
        }
    }
}

// The same staging by cp.async: every row's copies are in flight at once and
// the caller waits once (cp_async_wait_all, then a barrier).
template <int NT>
__device__ __forceinline__ void stage_rows_async(float4 *rows, const float *const *rptr, int nrows4,
                                                 int d0, int dc4) {
    constexpr int NW = NT / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int f = lane; f - lane < dc4; f += 32) {
        if (f >= dc4) continue;
        for (int r = warp; r < nrows4; r += NW)
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(static_cast<uint32_t>(
                             __cvta_generic_to_shared(&rows[srow4(r) + f]))),
                         "l"(rptr[r] + d0 + 4 * f)
                         : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

__device__ __forceinline__ void stage(const Smem &s, int nrows4, int d0, int dc4) {
    stage_rows<kThreads>(s.rows, s.rptr, nrows4, d0, dc4);
}

// Block bitonic sort of (pd, pid, prow) by (distance, id) over npad entries.
__device__ void sort_pool(const Smem &s, int npad) {
    const int tid = threadIdx.x;
    for (int k = 2; k <= npad; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int x = tid; x < npad; x += kThreads) {
                const int y = x ^ j;
                if (y > x) {
                    const bool up = (x & k) == 0;
                    if (lex_less(s.pd[y], s.pid[y], s.pd[x], s.pid[x]) == up) {
                        float td = s.pd[x]; s.pd[x] = s.pd[y]; s.pd[y] = td;
                        int32_t ti = s.pid[x]; s.pid[x] = s.pid[y]; s.pid[y] = ti;
                        ti = s.prow[x]; s.prow[x] = s.prow[y]; s.prow[y] = ti;
                    }
                }
            }
            __syncthreads();
        }
    }
}

template <int kNBF>
__global__ void __launch_bounds__(kThreads) prune_kernel(const PruneArgs a, int rows_cap,
                                                         int pool_cap, int slow_ok, int chunk,
                                                         const int32_t *idx_list,
                                                         const unsigned long long *idx_count) {
    extern __shared__ __align__(16) unsigned char smem[];
    Smem s;
    carve(smem, rows_cap, pool_cap, a.R, slow_ok != 0, s);
    __shared__ int64_t sh_i;  // first owner of the claimed chunk
    __shared__ int sh_np, sh_nk, sh_ebase;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int dim = a.dim;
    const int R = a.R;
    const int metric = a.metric;

    // owners: all of [0, n_owners), or the listed ones (pools the small-pool kernel passed on)
    const int64_t n_items = idx_list ? (int64_t)*idx_count : a.n_owners;
    for (;;) {
        if (tid == 0) sh_i = atomicAdd(a.work, chunk);
        __syncthreads();
        const int64_t i0 = sh_i;
        if (i0 >= n_items) break;
        const int64_t i1 = min(n_items, i0 + chunk);
      for (int64_t it = i0; it < i1; ++it) {
        const int64_t i = idx_list ? (int64_t)idx_list[it] : it;
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
        // 2. Drop -1, the owner and duplicates (first occurrence survives);
        //    the order of the survivors is irrelevant (they are sorted below).
        for (int j = tid; j < np_raw; j += kThreads) {
            const int32_t id = s.pid[j];
            bool ok = id >= 0 && id != owner;
            for (int t = 0; ok && t < j; ++t)
                if (s.pid[t] == id) ok = false;
            if (ok) s.tmp[atomicAdd(&sh_np, 1)] = id;
        }
        __syncthreads();
        const int np = sh_np;
        for (int j = tid; j < np; j += kThreads) {
            s.pid[j] = s.tmp[j];
            s.prow[j] = 1 + j;
        }
        int npad = 1;
        while (npad < np) npad <<= 1;
        for (int j = np + tid; j < npad; j += kThreads) {
            s.pd[j] = INFINITY;
            s.pid[j] = INT32_MAX;
            s.prow[j] = 0;
        }
        __syncthreads();

        int nk = 0;
        if (np <= kFastMax && 1 + np <= rows_cap) {
            // ---------------- fast path: one tile over owner + pool ----------------
            const int nrows = 1 + np;
            const int nB = (nrows + 3) >> 2;
            // a pool kept whole needs only the owner distances (block row 0)
            const bool whole = a.keep_all_if_fit && np <= R;
            const int nblk = whole ? nB : nB * (nB + 1) / 2;
            for (int r = tid; r < 4 * nB; r += kThreads)
                s.rptr[r] = seg_row(a.segs, r == 0 || r >= nrows ? owner : s.pid[r - 1], dim);
            // this thread's blocks (ba <= bb), enumerated row by row
            int bas[kNBF], bbs[kNBF];
#pragma unroll
            for (int t = 0; t < kNBF; ++t) {
                int b = tid + kThreads * t, ba = 0;
                if (b < nblk) {
                    while (b >= nB - ba) { b -= nB - ba; ++ba; }
                    bas[t] = ba;
                    bbs[t] = ba + b;
                } else {
                    bas[t] = -1;
                    bbs[t] = -1;
                }
            }
            f2_t acc[kNBF][4][4];
#pragma unroll
            for (int t = 0; t < kNBF; ++t)
#pragma unroll
                for (int p = 0; p < 4; ++p)
#pragma unroll
                    for (int q = 0; q < 4; ++q) acc[t][p][q] = 0ull;
            __syncthreads();
            for (int d0 = 0; d0 < dim; d0 += kDch) {
                const int dc4 = min(kDch, dim - d0) >> 2;
                stage(s, 4 * nB, d0, dc4);
                __syncthreads();
#pragma unroll
                for (int t = 0; t < kNBF; ++t) {
                    if (bas[t] < 0) continue;
                    const ulonglong2 *ra = reinterpret_cast<const ulonglong2 *>(s.rows + srow4(4 * bas[t]));
                    const ulonglong2 *rb = reinterpret_cast<const ulonglong2 *>(s.rows + srow4(4 * bbs[t]));
                    for (int f = 0; f < dc4; ++f) {
                        ulonglong2 xa[4], xb[4];
#pragma unroll
                        for (int p = 0; p < 4; ++p) {
                            xa[p] = ra[p * (kDch / 4 + 1) + f];
                            xb[p] = rb[p * (kDch / 4 + 1) + f];
                        }
#pragma unroll
                        for (int p = 0; p < 4; ++p)
#pragma unroll
                            for (int q = 0; q < 4; ++q)
                                acc[t][p][q] = chain2(acc[t][p][q], xa[p], xb[q], metric);
                    }
                }
                __syncthreads();
            }
            // the triangle replaces the staged rows
            float *T = reinterpret_cast<float *>(s.rows);
#pragma unroll
            for (int t = 0; t < kNBF; ++t) {
                if (bas[t] < 0) continue;
#pragma unroll
                for (int p = 0; p < 4; ++p)
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int ra = 4 * bas[t] + p, rb = 4 * bbs[t] + q;
                        if (ra < rb && rb < nrows) T[tri(ra, rb, nrows)] = chain2_final(acc[t][p][q], metric);
                    }
            }
            __syncthreads();
            for (int j = tid; j < np; j += kThreads) s.pd[j] = T[tri(0, 1 + j, nrows)];
            __syncthreads();
            sort_pool(s, npad);
            if (a.keep_all_if_fit && np <= R) {
                for (int j = tid; j < np; j += kThreads) s.kid[j] = s.pid[j];
                nk = np;
            } else {
                if (warp == 0) {
                    int nkk = 0;
                    for (int c = 0; c < np && nkk < R; ++c) {
                        const float dvc = s.pd[c];
                        const int cr = s.prow[c];
                        bool occ = false;
                        for (int j0 = 0; j0 < nkk && !occ; j0 += 32) {
                            const int j = j0 + lane;
                            bool t = false;
                            if (j < nkk) {
                                const int kr = s.krow[j];
                                const float dsc = kr < cr ? T[tri(kr, cr, nrows)] : T[tri(cr, kr, nrows)];
                                t = fmaf(a.alpha, dsc, -dvc) <= 0.f;
                            }
                            occ = __any_sync(0xffffffffu, t);
                        }
                        if (!occ) {
                            if (lane == 0) {
                                s.krow[nkk] = cr;
                                s.kid[nkk] = s.pid[c];
                            }
                            ++nkk;
                            __syncwarp();
                        }
                    }
                    if (lane == 0) sh_nk = nkk;
                }
                __syncthreads();
                nk = sh_nk;
            }
        } else {
            // ---------------- slow path: large pools ----------------
            // d(v, c): one thread per candidate, the same chain from global memory
            const float *orow = seg_row(a.segs, owner, dim);
            for (int j = tid; j < np; j += kThreads)
                s.pd[j] = prune_dist(orow, seg_row(a.segs, s.pid[j], dim), dim, metric);
            __syncthreads();
            sort_pool(s, npad);
            if (a.keep_all_if_fit && np <= R) {
                for (int j = tid; j < np; j += kThreads) s.kid[j] = s.pid[j];
                nk = np;
            } else {
                int pos = 0;
                while (pos < np && nk < R) {
                    const int cs = min(kTile, np - pos);
                    const int nrows = nk + cs;  // kept [0, nk), chunk [nk, nrows)
                    const int nA = (nrows + 3) >> 2, nB = (cs + 3) >> 2;
                    const int nblk = nA * nB;
                    for (int r = tid; r < 4 * nA; r += kThreads) {
                        const int32_t id = r < nk ? s.kid[r] : (r < nrows ? s.pid[pos + r - nk] : owner);
                        s.rptr[r] = seg_row(a.segs, id, dim);
                    }
                    for (int j = tid; j < nk; j += kThreads) s.krow[j] = j;
                    __syncthreads();
                    f2_t acc[kNBS][4][4];
#pragma unroll
                    for (int t = 0; t < kNBS; ++t)
#pragma unroll
                        for (int p = 0; p < 4; ++p)
#pragma unroll
                            for (int q = 0; q < 4; ++q) acc[t][p][q] = 0ull;
                    for (int d0 = 0; d0 < dim; d0 += kDch) {
                        const int dc4 = min(kDch, dim - d0) >> 2;
                        stage(s, 4 * nA, d0, dc4);
                        __syncthreads();
#pragma unroll
                        for (int t = 0; t < kNBS; ++t) {
                            const int b = tid + kThreads * t;
                            if (b >= nblk) continue;
                            const int ba = b / nB, bb = b - ba * nB;
                            const ulonglong2 *ra[4], *rb[4];
#pragma unroll
                            for (int p = 0; p < 4; ++p) {
                                ra[p] = reinterpret_cast<const ulonglong2 *>(s.rows + srow4(ba + nA * p));
                                int rbi = nk + bb + nB * p;
                                if (rbi >= 4 * nA) rbi = 0;
                                rb[p] = reinterpret_cast<const ulonglong2 *>(s.rows + srow4(rbi));
                            }
                            for (int f = 0; f < dc4; ++f) {
                                ulonglong2 xa[4], xb[4];
#pragma unroll
                                for (int p = 0; p < 4; ++p) {
                                    xa[p] = ra[p][f];
                                    xb[p] = rb[p][f];
                                }
#pragma unroll
                                for (int p = 0; p < 4; ++p)
#pragma unroll
                                    for (int q = 0; q < 4; ++q)
                                        acc[t][p][q] = chain2(acc[t][p][q], xa[p], xb[q], metric);
                            }
                        }
                        __syncthreads();
                    }
#pragma unroll
                    for (int t = 0; t < kNBS; ++t) {
                        const int b = tid + kThreads * t;
                        if (b >= nblk) continue;
                        const int ba = b / nB, bb = b - ba * nB;
#pragma unroll
                        for (int p = 0; p < 4; ++p)
#pragma unroll
                            for (int q = 0; q < 4; ++q) {
                                const int ar = ba + nA * p, bc = bb + nB * q;
                                if (ar < nrows && bc < cs && ar < nk + bc)
                                    s.stile[ar * kTile + bc] = chain2_final(acc[t][p][q], metric);
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
                                if (j < nkk)
                                    t = fmaf(a.alpha, s.stile[s.krow[j] * kTile + bc], -dvc) <= 0.f;
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
        }
        __syncthreads();

        // Output and reverse-edge emission.
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


// ---------------------------------------------------------------------------
// Small pools (at most 64 raw candidates: the source pool list(v) + c_cross
// results and most target pools).  128 threads, about 38 KB of shared memory:
// the owner row and every raw candidate row are staged once, one register-
// blocked pass builds the triangle of all pairwise distances (row 0 = the
// owner), all threads rank the candidates by (d(v,c), id) and build, for
// every candidate, the bitmask of earlier candidates that would occlude it;
// the greedy walk is then a loop over 64-bit masks.  The owner, -1 and
// duplicates (equal keys rank next to each other) are skipped.  Larger pools
// are appended to an overflow list for prune_kernel.

constexpr int kSmallThreads = 160;    // one 4x4 block of the triangle per thread
constexpr int kSmallMax = 64;
static_assert(kSmallMax == kPruneSmallMax, "the router sends pools of up to kSmallMax here");
constexpr int kSmallRows = 68;      // owner + 64, rounded up to 4
// distances of the (owner + pool) rows as a symmetric square matrix in the row
// buffer, row stride odd so a column read by 32 lanes hits 32 banks
constexpr int kSmallTs = 69;
static_assert(rows_float4(kSmallRows) * 4 >= (kSmallMax + 1) * kSmallTs, "matrix fits the row buffer");
constexpr int kSmallNB = 1;         // 17*18/2 = 153 blocks over 160 threads

struct SmallSmem {
    float4 rows[rows_float4(kSmallRows)];   // staged rows, then the distance matrix
    const float *rptr[kSmallRows];
    int32_t pid[kSmallMax];
    float kd[kSmallMax];       // raw keys
    int32_t kix[kSmallMax];
    float sd[kSmallMax];       // keys in (distance, id) order
    int32_t sid[kSmallMax];
    int32_t srow[kSmallMax];   // staged row of each ordered entry
    uint32_t occ[2 * kSmallMax];
};

#ifndef RNSM_SMALL_MIN_BLOCKS
#define RNSM_SMALL_MIN_BLOCKS 4   // resident CTAs per SM the register budget is cut for
#endif
// rows in flight per warp while the small-pool kernel stages its rows (more in
// flight spill registers of the 96 it has at four CTAs per SM)
#ifndef RNSM_SMALL_STAGE_UNROLL
#define RNSM_SMALL_STAGE_UNROLL 4
#endif
__global__ void __launch_bounds__(kSmallThreads, RNSM_SMALL_MIN_BLOCKS) prune_small_kernel(const PruneArgs a, int chunk) {
    __shared__ __align__(16) SmallSmem s;
    __shared__ int64_t sh_i;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int dim = a.dim;
    const int R = a.R;
    const int metric = a.metric;
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
        if (a.skip_empty_csr && c_hi == c_lo) continue;   // uniform: no shared state touched
        const int64_t nr_raw = (int64_t)a.lenA + a.lenB + (c_hi - c_lo);
        if (nr_raw > kSmallMax) {
            if (tid == 0) a.ovf_list[atomicAdd(a.ovf_count, 1ull)] = (int32_t)i;
            continue;
        }
        const int nr = (int)nr_raw;
        const float *orow = seg_row(a.segs, owner, dim);
        for (int j = tid; j < kSmallMax; j += kSmallThreads) {
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
            s.rptr[1 + j] = id >= 0 ? seg_row(a.segs, id, dim) : orow;
        }
        for (int r = kSmallMax + 1 + tid; r < kSmallRows; r += kSmallThreads) s.rptr[r] = orow;
        if (tid == 0) s.rptr[0] = orow;
        __syncthreads();

        const bool whole = a.keep_all_if_fit && nr <= R;
        const int nrows = 1 + nr;
        const int nB = (nrows + 3) >> 2;
        const int nblk = whole ? nB : nB * (nB + 1) / 2;
        int bas[kSmallNB], bbs[kSmallNB];
#pragma unroll
        for (int t = 0; t < kSmallNB; ++t) {
            int b = tid + kSmallThreads * t, ba = 0;
            if (b < nblk) {
                while (b >= nB - ba) { b -= nB - ba; ++ba; }
                bas[t] = ba;
                bbs[t] = ba + b;
            } else {
                bas[t] = -1;
                bbs[t] = -1;
            }
        }
        f2_t acc[kSmallNB][4][4];
#pragma unroll
        for (int t = 0; t < kSmallNB; ++t)
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[t][p][q] = 0ull;
        for (int d0 = 0; d0 < dim; d0 += kDch) {
            const int dc4 = min(kDch, dim - d0) >> 2;
            stage_rows_async<kSmallThreads>(s.rows, s.rptr, 4 * nB, d0, dc4);
            cp_async_wait_all();
            __syncthreads();
#pragma unroll
            for (int t = 0; t < kSmallNB; ++t) {
                if (bas[t] < 0) continue;
                const ulonglong2 *ra = reinterpret_cast<const ulonglong2 *>(s.rows + srow4(4 * bas[t]));
                const ulonglong2 *rb = reinterpret_cast<const ulonglong2 *>(s.rows + srow4(4 * bbs[t]));
                for (int f = 0; f < dc4; ++f) {
                    ulonglong2 xa[4], xb[4];
#pragma unroll
                    for (int p = 0; p < 4; ++p) {
                        xa[p] = ra[p * (kDch / 4 + 1) + f];
                        xb[p] = rb[p * (kDch / 4 + 1) + f];
                    }
#pragma unroll
                    for (int p = 0; p < 4; ++p)
#pragma unroll
                        for (int q = 0; q < 4; ++q)
                            acc[t][p][q] = chain2(acc[t][p][q], xa[p], xb[q], metric);
                }
            }
            __syncthreads();
        }
        float *T = reinterpret_cast<float *>(s.rows);
#pragma unroll
        for (int t = 0; t < kSmallNB; ++t) {
            if (bas[t] < 0) continue;
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int ra = 4 * bas[t] + p, rb = 4 * bbs[t] + q;
                    if (ra < rb && rb < nrows) {   // symmetric square layout
                        const float dv = chain2_final(acc[t][p][q], metric);
                        T[ra * kSmallTs + rb] = dv;
                        T[rb * kSmallTs + ra] = dv;
                    }
                }
        }
        __syncthreads();

        // Order: every raw entry's rank by (d(v,c), id), counted by all
        // threads; duplicates (equal keys) rank by raw index, so they land
        // next to each other; -1 and the owner sort last.
        for (int j = tid; j < kSmallMax; j += kSmallThreads) {
            const bool valid = j < nr && s.pid[j] >= 0;
            s.kd[j] = valid ? T[1 + j] : INFINITY;
            s.kix[j] = valid ? s.pid[j] : INT32_MAX;
        }
        __syncthreads();
        for (int j = tid; j < nr; j += kSmallThreads) {
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
        // Occluders of every candidate, in parallel: bit s of occ[c] (s < c in
        // the order) is set iff fmaf(alpha, d(s,c), -d(v,c)) <= 0.
        for (int c = warp; c < nr; c += kSmallThreads / 32) {
            const float dvc = s.sd[c];
            const int cr = s.srow[c];
            bool t0 = false, t1 = false;
            if (lane < c) {
                const int sr = s.srow[lane];
                t0 = fmaf(a.alpha, T[sr * kSmallTs + cr], -dvc) <= 0.f;
            }
            if (lane + 32 < c) {
                const int sr = s.srow[lane + 32];
                t1 = fmaf(a.alpha, T[sr * kSmallTs + cr], -dvc) <= 0.f;
            }
            const unsigned m0 = __ballot_sync(0xffffffffu, t0);
            const unsigned m1 = __ballot_sync(0xffffffffu, t1);
            if (lane == 0) {
                s.occ[2 * c] = m0;
                s.occ[2 * c + 1] = m1;
            }
        }
        __syncthreads();

        if (warp != 0 && i + 1 < i1) {
            // while warp 0 walks, the other warps bring the next owner's rows into L2
            const int64_t in = i + 1;
            const int32_t on = a.owner_ids ? a.owner_ids[in] : (int32_t)(a.owner_base + in);
            int64_t cl = 0, ch = 0;
            if (a.csr_offs) {
                cl = a.csr_offs[in];
                ch = a.csr_offs[in + 1];
            }
            const int64_t nrn = (int64_t)a.lenA + a.lenB + (ch - cl);
            if (nrn <= kSmallMax && !(a.skip_empty_csr && ch == cl)) {
                for (int j = tid - 32; j <= nrn; j += kSmallThreads - 32) {
                    int32_t id = on;   // j == nrn: the owner
                    if (j < nrn) {
                        if (j < a.lenA) {
                            id = a.listA[(int64_t)on * a.lenA + j];
                        } else if (j < a.lenA + a.lenB) {
                            id = a.listB[in * a.strideB + (j - a.lenA)];
                            if (id >= 0) id += a.offB;
                        } else {
                            id = a.csr_ids[cl + (j - a.lenA - a.lenB)];
                        }
                    }
                    if (id < 0) continue;
                    const char *row = reinterpret_cast<const char *>(seg_row(a.segs, id, dim));
                    for (int l = 0; l < dim * 4; l += 128) prefetch_l2(row + l);
                }
            }
        }

        if (warp == 0) {
            // live positions: valid and not a repeat of the previous id
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
                // The greedy walk in rounds: a position is decided once every live
                // occluder before it is; it is kept iff none of those is kept.  Each
                // decision depends only on earlier positions, so this is the walk's
                // uncapped kept set; the walk's cap keeps its first R positions.
                // Lane l holds positions l and l + 32.
                const unsigned long long oc0 =
                    lane < nr ? ((unsigned long long)s.occ[2 * lane] |
                                 ((unsigned long long)s.occ[2 * lane + 1] << 32)) & live : 0ull;
                const unsigned long long oc1 =
                    lane + 32 < nr ? ((unsigned long long)s.occ[2 * (lane + 32)] |
                                      ((unsigned long long)s.occ[2 * (lane + 32) + 1] << 32)) & live
                                   : 0ull;
                const unsigned long long b0 = 1ull << lane, b1 = 1ull << (lane + 32);
                unsigned long long decided = ~live, kall = 0ull;   // non-live: never kept
                while (~decided) {
                    // dropped as soon as one occluder is kept; kept once every occluder
                    // is decided and none is kept
                    const bool d0 = !(decided & b0), d1 = !(decided & b1);
                    const bool k0 = d0 && !(oc0 & kall) && !(oc0 & ~decided);
                    const bool k1 = d1 && !(oc1 & kall) && !(oc1 & ~decided);
                    const bool r0 = k0 || (d0 && (oc0 & kall));
                    const bool r1 = k1 || (d1 && (oc1 & kall));
                    decided |= (unsigned long long)__ballot_sync(0xffffffffu, r0) |
                               ((unsigned long long)__ballot_sync(0xffffffffu, r1) << 32);
                    kall |= (unsigned long long)__ballot_sync(0xffffffffu, k0) |
                            ((unsigned long long)__ballot_sync(0xffffffffu, k1) << 32);
                }
                while (__popcll(kall) > R) kall &= ~(1ull << (63 - __clzll((long long)kall)));
                kept = kall;
                nk = __popcll(kall);
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
        __syncthreads();
      }
        __syncthreads();  // every thread has read sh_i before it is claimed again
    }
}


// ---------------------------------------------------------------------------
// The greedy walk over kept rows only (pools of at most 64 raw candidates,
// dim <= 128).  The walk needs d(s, c) only for a kept s before c: the
// lowest open position (live, not yet occluded) is always kept, because
// every kept position before it has been tested against it.  So the walk
// goes kept row by kept row and tests each against the open positions after
// it -- on SIFT-like source pools about 900 of the 2,080 pair distances of
// the full triangle.  One CTA of 64 threads per owner; after ranking,
// thread t holds the row of position t in registers and every row sits in
// shared memory in position order, so the rows tested against are read as
// broadcasts.  Each round takes the first kWalkB open positions at once
// (kWalkB independent distance chains per thread): the first is kept, a
// later one is kept iff none of the kept ones before it occludes it (their
// mutual distances are among those computed), and the positions after the
// batch drop what the kept ones occlude.  Distances by a dropped member of
// the batch are discarded.  Every distance is the FP32 chain of the
// triangle kernel (a pair's order does not change it), so the kept lists
// are identical.
constexpr int kWalkThreads = 64;
// kF4: float4 of a row held in registers (16, 24 or 32: d <= 64, 96, 128); the
// row stride in shared memory is kF4 + 1 float4, so 8 rows fall on 32 banks
template <int kF4>
constexpr int walk_min_blocks() { return kF4 <= 16 ? 8 : kF4 <= 24 ? 6 : 5; }
#ifndef RNSM_WALK_B
#define RNSM_WALK_B 4
#endif
constexpr int kWalkB = RNSM_WALK_B;
#ifndef RNSM_WALK_CHUNK
#define RNSM_WALK_CHUNK 4   // source-pool owners per claim (4: 13.30 ms, 8: 13.35, 16: 13.44 on S6)
#endif

template <int kF4>
struct WalkSmem {
    float4 rows[kSmallMax * (kF4 + 1)];     // candidate rows in position order
    float4 vrow[kF4];                       // the owner's row
    float kd[kSmallMax];                    // raw keys
    int32_t kix[kSmallMax];
    int32_t sid[kSmallMax];                 // ids in position order
    float sd[kSmallMax];                    // d(v, c) in position order
    uint32_t occ[2][kWalkB][2];             // a round's occluded positions, per warp
    int64_t claim;
};

template <int kMetric, int kF4>
__global__ void __launch_bounds__(kWalkThreads, walk_min_blocks<kF4>())
    prune_walk_kernel(const PruneArgs a, int chunk) {
    constexpr int kWalkMaxF4 = kF4, kWalkStride = kF4 + 1;
    __shared__ __align__(16) WalkSmem<kF4> s;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int dim = a.dim, F4 = dim >> 2;
    const int R = a.R;
    // this thread's candidate row; the next owner's is loaded into it at the end
    // of an owner's walk, so its latency overlaps the output and the claim
    float4 xr[kWalkMaxF4];
    int64_t pre_i = -1;     // owner index whose candidate row xr already holds
    int32_t pre_id = -1;    // that candidate's id
    for (;;) {
        if (tid == 0) s.claim = atomicAdd(a.work, chunk);
        __syncthreads();
        const int64_t i0 = s.claim;
        __syncthreads();   // every thread has read the claim
        if (i0 >= a.n_owners) break;
        const int64_t i1 = min(a.n_owners, i0 + chunk);
        for (int64_t i = i0; i < i1; ++i) {
            const int32_t owner = a.owner_ids ? a.owner_ids[i] : (int32_t)(a.owner_base + i);
            int64_t c_lo = 0, c_hi = 0;
            if (a.csr_offs) {
                c_lo = a.csr_offs[i];
                c_hi = a.csr_offs[i + 1];
            }
            if (a.skip_empty_csr && c_hi == c_lo) continue;   // uniform
            const int64_t nr_raw = (int64_t)a.lenA + a.lenB + (c_hi - c_lo);
            if (nr_raw > kSmallMax) {
                if (tid == 0) a.ovf_list[atomicAdd(a.ovf_count, 1ull)] = (int32_t)i;
                continue;
            }
            const int nr = (int)nr_raw;
            // 1. raw candidate tid: its row into registers, the owner's row to
            //    shared memory, the candidate's key (d(v,c), id)
            int32_t id = -1;
            const bool have = pre_i == i;
            if (have) {
                id = pre_id;
            } else if (tid < nr) {
                if (tid < a.lenA) {
                    id = a.listA[(int64_t)owner * a.lenA + tid];
                } else if (tid < a.lenA + a.lenB) {
                    id = a.listB[i * a.strideB + (tid - a.lenA)];
                    if (id >= 0) id += a.offB;
                } else {
                    id = a.csr_ids[c_lo + (tid - a.lenA - a.lenB)];
                }
                if (id == owner) id = -1;
            }
            const float *orow = seg_row(a.segs, owner, dim);
            if (tid < F4) s.vrow[tid] = ldg4(orow + 4 * tid);
            if (!have) {
                const float *row = seg_row(a.segs, id >= 0 ? id : owner, dim);
#pragma unroll
                for (int f = 0; f < kWalkMaxF4; ++f)
                    if (f < F4) xr[f] = ldg4(row + 4 * f);
            }
            __syncthreads();
            {
                f2_t acc = 0ull;
#pragma unroll
                for (int f = 0; f < kWalkMaxF4; ++f)
                    if (f < F4)
                        acc = chain2(acc, *reinterpret_cast<const ulonglong2 *>(&s.vrow[f]),
                                     *reinterpret_cast<const ulonglong2 *>(&xr[f]), kMetric);
                const bool valid = tid < nr && id >= 0;
                s.kd[tid] = valid ? chain2_final(acc, kMetric) : INFINITY;
                s.kix[tid] = valid ? id : INT32_MAX;
            }
            __syncthreads();
            // 2. position = rank by (d(v,c), id); duplicates (equal keys) rank by
            //    raw index, so they land next to each other; -1 and the owner
            //    last.  The row moves to its position's slot.
            float my_dvc = 0.f;
            if (tid < nr) {
                const float dj = s.kd[tid];
                const int32_t ij = s.kix[tid];
                int r = 0;
                for (int k = 0; k < nr; ++k) {
                    const float dk = s.kd[k];
                    const int32_t ik = s.kix[k];
                    r += lex_less(dk, ik, dj, ij) || (dk == dj && ik == ij && k < tid);
                }
                s.sid[r] = ij;
                s.sd[r] = dj;
                float4 *dst = s.rows + r * kWalkStride;
#pragma unroll
                for (int f = 0; f < kWalkMaxF4; ++f)
                    if (f < F4) dst[f] = xr[f];
            }
            __syncthreads();
            if (tid < nr) {
                const float4 *src = s.rows + tid * kWalkStride;
#pragma unroll
                for (int f = 0; f < kWalkMaxF4; ++f)
                    if (f < F4) xr[f] = src[f];
                my_dvc = s.sd[tid];
            }
            // live positions: valid and not a repeat of the previous id
            unsigned long long live;
            {
                const bool a0 = lane < nr && s.sid[lane] != INT32_MAX &&
                                (lane == 0 || s.sid[lane - 1] != s.sid[lane]);
                const bool a1 = lane + 32 < nr && s.sid[lane + 32] != INT32_MAX &&
                                s.sid[lane + 31] != s.sid[lane + 32];
                live = (unsigned long long)__ballot_sync(0xffffffffu, a0) |
                       ((unsigned long long)__ballot_sync(0xffffffffu, a1) << 32);
            }
            unsigned long long kept = 0ull;
            if (a.keep_all_if_fit && __popcll(live) <= R) {
                kept = live;
            } else {
                // 3. the walk, kWalkB open positions per round
                unsigned long long open = live;
                int nk = 0, par = 0;
                while (open && nk < R) {
                    int p[kWalkB];
                    {
                        unsigned long long rest = open;
#pragma unroll
                        for (int b = 0; b < kWalkB; ++b) {
                            p[b] = rest ? __ffsll((long long)rest) - 1 : -1;
                            rest &= rest - 1ull;
                        }
                    }
                    // occlusion of this thread's position by each batch member
                    // before it; a warp with no open position after p[0] skips
                    const unsigned long long after = open & ~((2ull << p[0]) - 1ull);
                    const unsigned wopen = (unsigned)(after >> (32 * warp));
                    bool oc[kWalkB];
#pragma unroll
                    for (int b = 0; b < kWalkB; ++b) oc[b] = false;
                    if (wopen) {
                        f2_t acc[kWalkB];
                        const float4 *kr[kWalkB];
#pragma unroll
                        for (int b = 0; b < kWalkB; ++b) {
                            acc[b] = 0ull;
                            kr[b] = s.rows + (p[b] >= 0 ? p[b] : 0) * kWalkStride;
                        }
#pragma unroll
                        for (int f = 0; f < kWalkMaxF4; ++f) {
                            if (f < F4) {
                                const ulonglong2 x = *reinterpret_cast<const ulonglong2 *>(&xr[f]);
#pragma unroll
                                for (int b = 0; b < kWalkB; ++b)
                                    acc[b] = chain2(acc[b], *reinterpret_cast<const ulonglong2 *>(&kr[b][f]), x, kMetric);
                            }
                        }
                        const bool mine_open = (open >> tid) & 1ull;
#pragma unroll
                        for (int b = 0; b < kWalkB; ++b)
                            oc[b] = mine_open && p[b] >= 0 && p[b] < tid &&
                                    fmaf(a.alpha, chain2_final(acc[b], kMetric), -my_dvc) <= 0.f;
                    }
#pragma unroll
                    for (int b = 0; b < kWalkB; ++b) {
                        const unsigned m = __ballot_sync(0xffffffffu, oc[b]);
                        if (lane == 0) s.occ[par][b][warp] = m;
                    }
                    __syncthreads();
                    // resolve the batch in order
                    unsigned long long drop = 0ull;
#pragma unroll
                    for (int b = 0; b < kWalkB; ++b) {
                        if (p[b] < 0 || nk == R) break;
                        const unsigned long long bit = 1ull << p[b];
                        if (drop & bit) continue;   // occluded by a kept member
                        kept |= bit;
                        ++nk;
                        drop |= (unsigned long long)s.occ[par][b][0] |
                                ((unsigned long long)s.occ[par][b][1] << 32);
                    }
                    // everything up to the last member is decided
                    const int plast = p[kWalkB - 1] >= 0 ? p[kWalkB - 1] : 63;
                    open &= ~drop & ~((2ull << plast) - 1ull);   // 2 << 63 wraps to 0: all
                    par ^= 1;
                }
            }
            // the next owner of the claim: its candidate's row into xr now (the
            // walk is done with it); the same ids and rows as its own phase 1 loads
            pre_i = -1;
            if (i + 1 < i1) {
                const int64_t in = i + 1;
                const int32_t on = a.owner_ids ? a.owner_ids[in] : (int32_t)(a.owner_base + in);
                int64_t cl = 0, ch = 0;
                if (a.csr_offs) {
                    cl = a.csr_offs[in];
                    ch = a.csr_offs[in + 1];
                }
                const int64_t nrn = (int64_t)a.lenA + a.lenB + (ch - cl);
                if (!(a.skip_empty_csr && ch == cl) && nrn <= kSmallMax) {
                    int32_t idn = -1;
                    if (tid < nrn) {
                        if (tid < a.lenA) {
                            idn = a.listA[(int64_t)on * a.lenA + tid];
                        } else if (tid < a.lenA + a.lenB) {
                            idn = a.listB[in * a.strideB + (tid - a.lenA)];
                            if (idn >= 0) idn += a.offB;
                        } else {
                            idn = a.csr_ids[cl + (tid - a.lenA - a.lenB)];
                        }
                        if (idn == on) idn = -1;
                    }
                    const float *row = seg_row(a.segs, idn >= 0 ? idn : on, dim);
#pragma unroll
                    for (int f = 0; f < kWalkMaxF4; ++f)
                        if (f < F4) xr[f] = ldg4(row + 4 * f);
                    pre_i = in;
                    pre_id = idn;
                }
            }
            // 4. output in (distance, id) order: the kept positions
            if (warp == 0) {
                const int nk = __popcll(kept);
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
            __syncthreads();   // the owner's shared state is free
        }
    }
}

}  // namespace

// The general FP32 prune (any pool up to 4,096 raw candidates); with idx_list,
// only the listed owner indices (idx_count of them, read on the device).
cudaError_t launch_prune_general(const PruneArgs &a, const int32_t *idx_list,
                           const unsigned long long *idx_count, cudaStream_t st) {
    const int64_t maxpool = (int64_t)a.lenA + a.lenB + (a.csr_offs ? a.csr_max : 0);
    int pool_cap = 64;
    while (pool_cap < maxpool && pool_cap < kPoolCapMax) pool_cap <<= 1;
    const bool slow = maxpool > kFastMax;
    const int fast_rows = 4 * (int)((std::min<int64_t>(maxpool, kFastMax) + 1 + 3) / 4);
    const int slow_rows = 4 * ((a.R + kTile + 3) / 4);
    const int rows_cap = slow ? std::max(fast_rows, slow_rows) : fast_rows;
    const size_t smem = smem_bytes(rows_cap, pool_cap, a.R, slow);
    auto kern = fast_rows <= kRowsNB1 ? prune_kernel<1> : prune_kernel<kNBFMax>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    int64_t grid = (int64_t)sms * per_sm;
    // Sparse passes (most owners without CSR entries) claim owners 32 at a time.
    const int chunk = a.skip_empty_csr && !idx_list ? 32 : 1;
    if (!idx_list) {
        const int64_t want = (a.n_owners + chunk - 1) / chunk;
        if (want < grid) grid = want;
    }
    kern<<<(unsigned)grid, kThreads, smem, st>>>(a, rows_cap, pool_cap, slow ? 1 : 0, chunk,
                                                 idx_list, idx_count);
    note_launches(1);
    return cudaGetLastError();
}

namespace {

template <int kMetric, int kF4>
cudaError_t launch_walk_t(const PruneArgs &a, cudaStream_t st) {
    auto kern = prune_walk_kernel<kMetric, kF4>;
    cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kWalkThreads, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    // owners per claim: the next owner's rows are loaded during the current one's
    // walk only within a claim
    const int chunk = a.skip_empty_csr ? 8 : RNSM_WALK_CHUNK;
    int64_t grid = (int64_t)sms * per_sm;
    const int64_t want = (a.n_owners + chunk - 1) / chunk;
    if (want < grid) grid = want;
    kern<<<(unsigned)grid, kWalkThreads, 0, st>>>(a, chunk);
    note_launches(1);
    return cudaGetLastError();
}

template <int kMetric>
cudaError_t launch_walk_m(const PruneArgs &a, cudaStream_t st) {
    if (a.dim <= 64) return launch_walk_t<kMetric, 16>(a, st);
    if (a.dim <= 96) return launch_walk_t<kMetric, 24>(a, st);
    return launch_walk_t<kMetric, 32>(a, st);
}

}  // namespace

cudaError_t launch_walk(const PruneArgs &a, cudaStream_t st) {
    static_assert(4 * 32 == kPruneWalkMaxDim, "rows held in registers");
    if (a.dim > kPruneWalkMaxDim) return cudaErrorInvalidValue;
    return a.metric == 0 ? launch_walk_m<0>(a, st) : launch_walk_m<1>(a, st);
}

cudaError_t launch_small(const PruneArgs &a, cudaStream_t st) {
    cudaError_t e;
    cudaFuncSetAttribute(prune_small_kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, prune_small_kernel, kSmallThreads, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    // owners are claimed a few at a time: one atomic round trip per claim
    const int chunk = a.skip_empty_csr ? 8 : 4;
    int64_t grid = (int64_t)sms * per_sm;
    const int64_t want = (a.n_owners + chunk - 1) / chunk;
    if (want < grid) grid = want;
    prune_small_kernel<<<(unsigned)grid, kSmallThreads, 0, st>>>(a, chunk);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace rnsm
