// Internal launchers shared by the translation units of librnsm.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace rnsm {

// Sets the calling thread's rnsm_last_error() message.
void set_last_error(const char *msg);

// Kernels launched by this library (every launcher adds its count).
void note_launches(int n);
long long launches_so_far();

enum SeedMode : int32_t { kSeedConst = 0, kSeedSelf = 1, kSeedTable = 2 };

// One (source, target) pair of a multi-job search launch: its fields replace
// those of the same names in SearchArgs for the queries
// [q_begin, next job's q_begin) of the launch.
struct SearchJob {
    const float *base;
    const int32_t *adj;
    const float *qvecs;
    const int32_t *qidx;
    const int32_t *seed_tab;
    const int32_t *seed_row;
    int32_t *out_ids;
    int64_t q_begin;
    int64_t n_base;
    int32_t r_in;
    int32_t seed_const;
    int32_t id_offset;
    int32_t pad;
};

// One batched beam-search launch (Algorithm 1).  Query i of the launch is
// query g = q0 + i of the batch; it reads qvecs[qrow * dim] with
// qrow = qidx ? qidx[g] : g.  With a job table (jobs, device memory,
// n_jobs + 1 entries, the last one a sentinel whose q_begin is the total),
// g selects the job and counts from the job's q_begin; nq is the total.
struct SearchArgs {
    const float *base;      // searched vector set [n_base * dim]
    int64_t n_base;
    const int32_t *adj;     // [n_base * r_in]
    int32_t r_in;
    int32_t dim;
    int32_t metric;
    const float *qvecs;
    const int32_t *qidx;    // nullable
    int64_t nq;
    int64_t q0;             // query i of this launch is query q0 + i of the batch
    int32_t seed_mode;      // SeedMode
    int32_t seed_const;     // kSeedConst: the single entry vertex
    const int32_t *seed_tab;  // kSeedTable: rows of seeds
    int32_t seed_stride;
    int32_t n_seeds;
    const int32_t *seed_row;  // kSeedTable: row = seed_row ? seed_row[qrow] : i
    int32_t ef;
    int32_t k;
    int32_t exclude_self;     // drop result id == qrow (neighbour expansion)
    int32_t *out_ids;         // row = out_by_qidx ? qrow : i
    int32_t out_stride;
    int32_t out_by_qidx;
    int32_t id_offset;        // added to every written id
    float *out_d;             // nullable, same layout as out_ids
    int64_t *out_ndc;         // nullable, [nq]
    unsigned long long *stats;  // nullable: [0] += NDC, [1] += expansions
    int32_t *work;            // zeroed work counter
    const SearchJob *jobs;    // nullable: multi-job launch (out_d and out_ndc unused)
    int32_t n_jobs;
};

cudaError_t launch_search(const SearchArgs &a, cudaStream_t st);
cudaError_t launch_search_jobs(const SearchArgs &a, int var, cudaStream_t st);
// True if a launch of nq queries would run the autotuner (timed chunks, host waits).
bool search_would_tune(int dim, int ef, int seed_mode, int64_t nq);

// Occlusion prune (UpdateGraph) of a batch of owners over a segment table.
// Owner i is global id owner_ids ? owner_ids[i] : owner_base + i.  Its pool
// is the union of: listA row gid (lenA ids), listB row i (lenB ids, offB
// added to non-negative ones), CSR row i (csr_offs/csr_ids).
struct PruneArgs {
    SegTable segs;
    int32_t dim;
    int32_t metric;
    float alpha;
    int32_t R;
    int32_t keep_all_if_fit;
    int32_t skip_empty_csr;   // owners with no CSR entries are left untouched
    int64_t n_owners;
    const int32_t *owner_ids;
    int32_t owner_base;
    const int32_t *listA;
    int32_t lenA;
    const int32_t *listB;
    int32_t strideB;
    int32_t lenB;
    int32_t offB;
    const int64_t *csr_offs;
    const int32_t *csr_ids;
    int32_t csr_max;          // longest CSR row (sizes the pool buffer)
    int32_t *out;             // rows by owner gid (out_by_index: by i), stride R
    int32_t out_by_index;
    int32_t emit_lo, emit_hi; // kept ids in [emit_lo, emit_hi) emit (u, owner)
    int32_t *eu;
    int32_t *ev;
    unsigned long long *ecount;
    int32_t prec;             // 0 FP32; 1 BF16 / 2 FP8 tiles on the tensor cores
    const void *qrows;        // quantized rows by global id [N * dim] (BF16 or E4M3)
    const void *qrows_lo;     // nullable: BF16 low terms lo = bf16(x - hi), qrows holding hi
    const float *qscale;      // FP8 per-row scale
    const float *qerr;        // residual norms ||x - x~||
    const float *qnorm;       // row norms ||x||
    unsigned long long *rechecks;  // decisions re-decided in FP32
    unsigned long long *tile_tests;  // nullable: occlusion tests the tensor-core tiles evaluated
    int32_t tune_site;       // the prune autotuner's call site (0 any, 1 merge S6, 2 merge S7):
                             // pools of one shape differ between a graph build and a merge
    unsigned int *tile_err;   // nullable [4]: sampled tile error maxima (float bits) and count
    int32_t *work;
    int32_t *work2;           // second zeroed counter (overflow pass)
    int32_t *ovf_list;        // [n_owners]: owners whose pool exceeds the small-pool kernel
    unsigned long long *ovf_count;
    int32_t *err;             // bit 4: pool larger than the capacity; bit 6: tile wait ran out
    int32_t test_withhold_commit;  // test-only (tensor-core prune): never signal MMA completion
    int32_t pair_hi_only;     // pair tile: integer rows spanning <= 256, hi terms only
};

// variant (optional): set to the prune variant that served the call (0 the
// FP32 triangle, 1 the pair tile, 2 the general tile, 3 the FP32 walk).
cudaError_t launch_prune(const PruneArgs &a, cudaStream_t st, int *variant = nullptr);
// The FP32 kernels behind it: the small-pool kernel (raw pools of at most
// kPruneSmallMax; larger ones go to a->ovf_list) and the general kernel (with
// idx_list: only the listed owner indices, idx_count of them on the device).
constexpr int kPruneSmallMax = 64;
cudaError_t launch_small(const PruneArgs &a, cudaStream_t st);
// The same pools (d <= kPruneWalkMaxDim) by the walk over kept rows only.
constexpr int kPruneWalkMaxDim = 128;
cudaError_t launch_walk(const PruneArgs &a, cudaStream_t st);
cudaError_t launch_prune_general(const PruneArgs &a, const int32_t *idx_list,
                                 const unsigned long long *idx_count, cudaStream_t st);

// Tensor-core prune (BF16 / FP8 tiles with FP32 re-decisions) of pools up to
// prune_tc_max_pool() raw candidates.  prune_tc_terms: 0 if (dim, prec) has no
// tensor-core tile, 1 if it stages the quantized rows (qrows, qscale, qerr,
// qnorm), 2 if it stages the FP32 rows split into two BF16 terms.
// With the metric known, FP8 at inner product from d = 384 stages two E4M3
// terms (hi, lo, stored by launch_quantize with q_lo).
int prune_tc_terms(int dim, int prec, int metric = -1);
int prune_tc_max_pool();
cudaError_t launch_prune_tc(const PruneArgs &a, cudaStream_t st, int terms = 0);  // 0: prune_tc_terms
// BF16 tensor-core prune of small pools, two owners per tile (L2, dim a
// multiple of 16 up to 128, pools of up to prune_pair_max_pool() raw
// candidates; FP32 rows centred and split into hi / lo terms in the kernel,
// nothing stored).
bool prune_pair_ok(int dim, int prec, int metric);
int prune_pair_max_pool();
cudaError_t launch_prune_pair(const PruneArgs &a, cudaStream_t st);
// *hi_only = 1 if every component of the table's rows is an integer and they span
// at most 256 (scratch: 3 device ints; synchronises the stream).
cudaError_t launch_pair_exact_check(const SegTable &t, int32_t dim, int32_t *scratch, int32_t *hi_only,
                                    cudaStream_t st);
// Rows of the segment table to BF16 (prec 1) or E4M3 with per-row scale (prec 2),
// plus residual norms and row norms.
// With q_lo the rows are split into two terms, q = bf16(x) and q_lo = bf16(x - q),
// or for E4M3 q = e4m3(x / s) and q_lo = e4m3(x / s - q), and err is the norm of
// what is left.
cudaError_t launch_quantize(const SegTable &segs, int64_t n, int32_t dim, int prec, void *q,
                            void *q_lo, float *scale, float *err, float *norm, cudaStream_t st);

// The multi-pair union variant (union.cu).  UnionEdges: the plan edges of one
// source, in plan order: result rows (by local source vertex, L wide, local
// target ids) and the global offset of each target.  UnionMasks: per segment,
// the bit set of its targets (0: not a source of the plan).
struct UnionEdges {
    const int32_t *res[kMaxSeg];
    int32_t t0[kMaxSeg];
    int32_t n;
};
struct UnionMasks {
    unsigned long long tmask[kMaxSeg];
};
cudaError_t launch_union_pool(const UnionEdges &e, int64_t ns, int32_t L, int32_t c, int32_t *pool,
                              cudaStream_t st);
cudaError_t launch_emit_cross(const int32_t *lists, int32_t R, const SegTable &t, const UnionMasks &mk,
                              int32_t *eu, int32_t *ev, unsigned long long *count, cudaStream_t st);

// Query schedule (schedule.cu).  launch_locality_order: the n rows of x
// counting-sorted by a random-hyperplane locality key (order) and each row's
// position in that order (rank); keys, vals: n scratch entries each; offs,
// cursor, scan: counting-sort scratch for min(n, 4096) keys.
cudaError_t launch_locality_order(const float *x, int64_t n, int32_t dim, int32_t *keys,
                                  int32_t *vals, int64_t *offs, int32_t *cursor, void *scan_tmp,
                                  size_t scan_tmp_bytes, int32_t *order, int32_t *rank,
                                  cudaStream_t st);
// Pivots sorted by rank, followers by the rank of their pivot (counting-sort
// scratch for n keys); the order inside one pivot's followers is unspecified.
cudaError_t order_search_lists(const int32_t *rank, const int32_t *pivot_of, int32_t *pivots,
                               int64_t np, int32_t *followers, int64_t nf, int64_t n,
                               int32_t *keys, int32_t *vals, int64_t *offs, int32_t *cursor,
                               void *scan_tmp, size_t scan_tmp_bytes, cudaStream_t st);

// Counting sort of (key, val) pairs by key into CSR (K3).
// keys/vals [cap], the number of valid pairs at *count (device) or n_host.
cudaError_t launch_bucket(const int32_t *keys, const int32_t *vals, int64_t cap,
                          const unsigned long long *count, int64_t nkeys, int32_t key_offset,
                          int64_t *offs /*[nkeys+1]*/, int32_t *cursor /*[nkeys]*/,
                          int32_t *out_vals, void *scan_tmp, size_t scan_tmp_bytes,
                          cudaStream_t st);
size_t bucket_scan_tmp_bytes(int64_t nkeys);

// Sorts every CSR row ascending (rows of at most 4096 entries).
cudaError_t launch_sort_rows(const int64_t *offs, int32_t *ids, int64_t nrows, int32_t *err,
                             cudaStream_t st);

// (N+ first k columns) -> pairs (x, y) for the reverse-kNN inversion.
cudaError_t launch_rk_pairs(const int32_t *nplus, int64_t n, int32_t k_plus, int32_t k,
                            int32_t *keys, int32_t *vals, unsigned long long *count,
                            cudaStream_t st);

// *out = longest row of a CSR with n rows.
cudaError_t launch_max_row(const int64_t *offs, int64_t n, int32_t *out, cudaStream_t st);

bool search_dim_supported(int dim);

// S3 on the device (parallel rounds, same result as the lazy greedy).
// tmp: pivot_tmp_bytes(n); counters: 2 device u64.  Writes pivot_of [n]
// (-1 pivots), the pivot and follower lists (ascending-free order) and counts.
size_t pivot_tmp_bytes(int64_t n);
cudaError_t select_pivots_device(const int32_t *nplus, int64_t n, int32_t k_plus, int32_t k,
                                 const int64_t *offs, const int32_t *ids, int32_t *pivot_of,
                                 int32_t *pivots, int32_t *followers, int64_t *n_pivots,
                                 int64_t *n_followers, int32_t *rounds, void *tmp,
                                 unsigned long long *counters, cudaStream_t st);

cudaError_t launch_validate_graph(const int32_t *adj, int64_t n, int32_t r_in, int32_t *err,
                                  cudaStream_t st);
// Sets bit 1 of *err if an id is outside [allow_minus1 ? -1 : 0, bound).
cudaError_t launch_validate_ids(const int32_t *ids, int64_t count, int64_t bound,
                                int32_t allow_minus1, int32_t *err, cudaStream_t st);
cudaError_t launch_validate_vecs(const float *v, int64_t count, int32_t *err, cudaStream_t st);
cudaError_t launch_init_lists(const int32_t *adj, int64_t n, int32_t r_in, int32_t offset,
                              int32_t *out, int32_t R, cudaStream_t st);
cudaError_t launch_fill(int32_t *p, int64_t count, int32_t value, cudaStream_t st);
// Medoid: partial sums [nblk * dim] doubles, then argmin; result to *out (device).
cudaError_t launch_medoid(const float *v, int64_t n, int32_t dim, int32_t metric, double *tmp,
                          size_t tmp_bytes, int32_t *out, cudaStream_t st);
size_t medoid_tmp_bytes(int64_t n, int32_t dim);

}  // namespace rnsm
