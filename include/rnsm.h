/*
 * rnsm.h -- C ABI of the GB300 (sm_103a) implementation of Reverse Neighbor
 * Sliding Merge (RNSM) and Merge Order Selection (MOS), arxiv 2602.17099.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Pointers documented as "device" are CUDA device pointers on the current
 *   device; "host" pointers are ordinary CPU memory.  The caller owns every
 *   buffer it passes in.  Scratch memory is taken from a per-device workspace
 *   that the library grows on demand and keeps until rnsm_release_workspace()
 *   or process exit.
 * - Vectors are row-major float32, rows contiguous, 16-byte aligned (dim must
 *   be a multiple of 4, at most 1024).  Calls that search (rnsm_search,
 *   rnsm_expand, rnsm_build_segment, rnsm_merge) need a dimension the search
 *   kernel is built for: 8, 16, 32, 64, 96, 128, 256 or 768; the prune,
 *   reverse-edge and medoid calls take any.  The BF16 / FP8 prune tiles need
 *   dim a multiple of 16 (BF16) or 32 (FP8); other dimensions run the FP32
 *   kernels.  Graphs are int32 adjacency rows padded with -1.
 * - Timeouts: the tensor-core prune waits on its MMAs for at most one second;
 *   a wait that runs out ends the call with RNSM_ETIMEOUT, the context usable.
 * - Distances (native, never square-rooted): RNSM_METRIC_L2 = squared
 *   Euclidean distance (orders exactly like the paper's delta, notation table
 *   of Section 2); RNSM_METRIC_IP = 1 - <x, y> for unit-norm embeddings.
 * - Candidate order is (distance, id) ascending everywhere; ties go to the
 *   lower id.
 * - Every call is enqueued on `stream` (a cudaStream_t, NULL = legacy default
 *   stream) and blocks until its results are in the output buffers.
 * - Inputs are validated before any launch: bad sizes or parameters give
 *   RNSM_EINVAL, out-of-range vertex ids or non-finite vectors RNSM_EGRAPH.
 *   CUDA failures give RNSM_ECUDA.  rnsm_last_error() describes the last
 *   non-OK status of the calling thread.
 * - Autotuning: the first large search launch of a shape and the first large
 *   prune call of a shape time their kernel variants on slices of the call and
 *   keep the fastest for the process; every variant gives the same results.
 *   Environment variables read at each call (none changes a result):
 *     RNSM_SEARCH_VARIANT=v   force search launch variant v (0..3)
 *     RNSM_PRUNE_VARIANT=v    force prune variant v where it applies (0 the
 *                             FP32 triangle, 1 the pair tile, 2 the general
 *                             tile, 3 the FP32 walk)
 *     RNSM_TUNE_LOG=1|2       print the prune tuner's choices (2: and slices)
 *                             to stderr
 *     RNSM_SEARCH_PER_JOB=1   run a plan's multi-job searches as one launch
 *                             per plan edge (to measure the batched launches)
 *     RNSM_TEST_WITHHOLD_COMMIT  tests only: the tensor-core prune withholds
 *                             its MMA completion signal, so that its bounded
 *                             wait runs out (RNSM_ETIMEOUT)
 */
#ifndef RNSM_H_
#define RNSM_H_

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define RNSM_API __attribute__((visibility("default")))
#else
#define RNSM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    RNSM_OK = 0,
    RNSM_EINVAL = 1,   /* bad argument (size, parameter, pointer) */
    RNSM_ENOMEM = 2,   /* device or host allocation failed */
    RNSM_ECUDA = 3,    /* a CUDA call or kernel failed */
    RNSM_ETIMEOUT = 4, /* a bounded device wait ran out */
    RNSM_EGRAPH = 5    /* malformed graph or vector data */
} rnsm_status;

typedef enum { RNSM_METRIC_L2 = 0, RNSM_METRIC_IP = 1 } rnsm_metric;

/* Arithmetic of the candidate-by-candidate prune tiles (Section 4.2,
 * UpdateGraph).  Searches always run in FP32.  BF16 and FP8 tiles run on the
 * tensor cores and every decision a tile cannot settle within its error bound
 * is re-decided with the FP32 distance, so the result equals the FP32 one. */
typedef enum { RNSM_PREC_FP32 = 0, RNSM_PREC_BF16 = 1, RNSM_PREC_FP8 = 2 } rnsm_precision;

/* One input segment: a vector set X_i and its proximity graph G_i
 * (Problem Definition, Section 3.1). */
typedef struct {
    int64_t n;           /* number of vertices */
    int32_t dim;         /* vector dimension, multiple of 4, same for all segments */
    int32_t r_in;        /* adjacency row length (<= R of the merge) */
    const float *vecs;   /* device, [n * dim] */
    const int32_t *adj;  /* device, [n * r_in], local ids in [0, n), -1 padded */
    int32_t entry;       /* default entry vertex of G_i (local id) */
} rnsm_segment;

/* Merge parameters (Algorithm 2).  A zero field takes its default:
 * k_rev 5 (reverse k; the paper uses 3, 5, 7), k_plus max(2*k_rev, 16)
 * (expansion factor k+), ef_slide ceil(L/2) (local-sliding effort ef_L),
 * c_cross = ef_slide (search results that enter the prune); 1 <= c_cross <=
 * ef_slide <= L.
 * L is the naive-search effort ef_N; R the output degree; alpha the
 * occlusion factor of the prune (c is dropped when a kept s has
 * alpha * d(s, c) <= d(v, c)). */
typedef struct {
    int32_t R;
    int32_t L;
    float alpha;
    int32_t metric;      /* rnsm_metric */
    int32_t prec;        /* rnsm_precision of the prune tiles */
    int32_t k_rev;
    int32_t k_plus;
    int32_t ef_slide;
    int32_t c_cross;
    uint32_t flags;      /* RNSM_FLAG_* */
} rnsm_params;

/* Cross-query Merge comparator (Section 3.1): every source vertex runs a
 * naive search (no pivots, no sliding). */
#define RNSM_FLAG_CM 0x1u
/* Run pivot selection (S3) with the host lazy greedy instead of the device
 * rounds (identical results; for cross-checking). */
#define RNSM_FLAG_HOST_PIVOTS 0x2u
/* Capture the searches, prunes and reverse-edge updates of the plan (S4 to S7)
 * in a CUDA graph and replay it when the next call has the same inputs,
 * parameters, plan and pivot counts (identical results; the capture is used
 * once the search launch shapes are autotuned and the plan's result tables
 * fit one group).  phase_ms[4] then holds S4 to S7 together. */
#define RNSM_FLAG_GRAPH 0x4u
/* Multi-pair union variant (not in the paper; for merging several pairs at
 * once, e.g. several new partitions of an incremental merge): the searches
 * of every plan edge as in Algorithm 2, then ONE prune per source vertex of
 * its list and the first c_cross results of each of its plan edges (in plan
 * order), then ONE reverse-edge pass over the kept cross edges of every
 * source (a cross edge: one into a target segment of a plan edge of that
 * source).  Every prune sees the lists as they were before the plan's reverse
 * edges.  Needs the plan's result tables to fit one group (L * 4 bytes per
 * source vertex per edge, 4 GiB in all); not combined with RNSM_FLAG_GRAPH. */
#define RNSM_FLAG_UNION 0x8u

/* One edge of a merge plan: segment `src` is merged into segment `dst`.
 * Plan order = array order (Section 5: closer pairs first). */
typedef struct {
    int32_t src;
    int32_t dst;
    double cost;
} mos_edge;

typedef struct {
    double wall_s;         /* rnsm_merge entry to return */
    double host_pivot_s;   /* host time in pivot selection */
    int64_t ndc;           /* distance computations of all searches */
    int64_t expansions;    /* beam expansions of all searches */
    int64_t rechecks;      /* prune decisions re-decided in FP32 */
    int64_t pivots;        /* naive searches */
    int64_t followers;     /* local-sliding searches */
    int64_t reverse_edges; /* cross edges kept on the source side */
    int64_t launches;      /* CUDA kernels launched by the call */
    /* CUDA-event time per step on the call's stream, summed over plan edges:
     * [0] validation and list initialisation, [1] S1 expansion, [2] S2
     * inversion, [3] S3 pivot selection incl. its host copies, [4] S4 pivot
     * search, [5] S5 follower search, [6] S6 source prune, [7] S7 reverse
     * edges. */
    double phase_ms[8];
    int64_t search_ndc[3]; /* NDC of S1, S4, S5 */
    int64_t search_exp[3]; /* expansions of S1, S4, S5 */
    int64_t search_queries[3]; /* queries of S1, S4, S5 */
    /* BF16 / FP8 modes: distance error of the tensor-core prune tiles, sampled
     * on the owner distances of every 64th owner: [0] max |d~ - d64| / d64
     * (tile vs FP64), [1] max |d32 - d64| / d64 (the FP32 distance vs FP64),
     * [2] max |d~ - d32| / B (the share of its error bound B the tile used),
     * [3] number of distances sampled.  Zero in FP32 mode. */
    double tile_error[4];
    /* BF16 / FP8 modes: occlusion tests the tensor-core tiles evaluated (the
     * share that was re-decided is rechecks / tile_tests, owner-distance
     * re-decisions of the general tile included in rechecks).  Zero in FP32. */
    int64_t tile_tests;
    /* The prune kernel that served the last S6 call and the last S7 pool prune
     * (the autotuner's choice): 0 the FP32 register-blocked triangle, 1 the
     * pair tensor-core tile, 2 the general tensor-core tile, 3 the FP32 walk
     * over kept rows; -1 none ran, or the call replayed a captured CUDA graph
     * (RNSM_FLAG_GRAPH), whose kernels were chosen when it was captured. */
    int32_t prune_kernel[2];
} rnsm_stats;

/*
 * mos_plan -- Merge Order Selection, Algorithm 3 (Section 5), plus the
 * execution order of its edges (Section 5, after Algorithm 3).
 *   m                 number of segments (>= 1)
 *   sizes             host [m] vertex counts
 *   centroids         host [m * D] segment centroids, or NULL: unit cost for
 *                     every pair (random partitions).  Cost = Euclidean
 *                     distance between centroids.
 *   degree_bound      merge-graph degree bound R of Algorithm 3; 0 selects
 *                     ceil(sqrt(m - 1)) + 1
 *   diameter_bound    Delta of Algorithm 3; 0 selects 2
 *   out               host [*n_out capacity] edges, ascending cost (ties by
 *                     (min index, max index)), each oriented smaller segment
 *                     -> larger (equal sizes: larger index -> smaller)
 *   n_out             in: capacity of out; out: number of edges
 * Host only; no device work.  RNSM_EINVAL if the capacity is too small.
 */
RNSM_API rnsm_status mos_plan(int32_t m, const int64_t *sizes, const float *centroids, int32_t D,
                     int32_t degree_bound, int32_t diameter_bound, mos_edge *out,
                     int32_t *n_out);

/*
 * rnsm_merge -- RNSM over a plan of segment pairs (Algorithm 2, Section 4.2).
 * For each plan edge (s -> t), in order:
 *   S1 neighbour expansion of s (beam search in G_s seeded at each vertex),
 *   S2 reverse-kNN inversion R_k, S3 lazy-greedy pivot selection (host),
 *   S4 naive search of each pivot in the original G_t (ef = L),
 *   S5 local sliding of each follower seeded with its pivot's results
 *      (ef = ef_slide), S6 prune of list(v) + first c_cross results to R for
 *   every v in s, S7 reverse edges into t (pool <= R: kept as is, else pruned).
 * S1-S3 run once per source segment.
 *   segs, m       device segments (m >= 1, equal dim; sum n < 2^31)
 *   p             parameters (zeros -> defaults)
 *   plan, n_plan  host merge plan; plan == NULL with m == 2 merges the smaller
 *                 segment into the larger one (equal sizes: 1 -> 0)
 *   out_adj       device [N * R], N = sum of n; row v is the merged list of
 *                 global vertex v (global id = segment offset + local id in
 *                 segment order); lists touched by a prune are sorted by
 *                 (distance, id); untouched lists are the input lists.
 *   stream        cudaStream_t
 *   stats         host, nullable
 */
RNSM_API rnsm_status rnsm_merge(const rnsm_segment *segs, int32_t m, const rnsm_params *p,
                       const mos_edge *plan, int32_t n_plan, int32_t *out_adj, void *stream,
                       rnsm_stats *stats);

/* Bytes of device workspace rnsm_merge takes for these inputs. */
RNSM_API size_t rnsm_workspace_size(const rnsm_segment *segs, int32_t m, const rnsm_params *p);

/* Frees the calling device's workspace (after synchronising). */
RNSM_API void rnsm_release_workspace(void);

/*
 * rnsm_search -- batched AKNN beam search, Algorithm 1 (Section 2.2).
 *   vecs, n, dim, adj, r_in   device graph to search
 *   queries, nq               device [nq * dim]
 *   seeds, n_seeds            device [nq * n_seeds] entry vertices per query
 *                             (-1 = none); duplicates are evaluated once
 *   ef                        beam width (1..256); k <= ef results returned
 *   out_ids                   device [nq * k], (distance, id) order, -1 padded
 *   out_dists                 device [nq * k] or NULL (FP32 native distance)
 *   out_ndc                   device [nq] int64 distance-computation counts or NULL
 */
RNSM_API rnsm_status rnsm_search(const float *vecs, int64_t n, int32_t dim, const int32_t *adj,
                        int32_t r_in, const float *queries, int64_t nq, const int32_t *seeds,
                        int32_t n_seeds, int32_t ef, int32_t k, int32_t metric,
                        int32_t *out_ids, float *out_dists, int64_t *out_ndc, void *stream);

/*
 * rnsm_expand -- ExpandNeighbors of Algorithm 2 (Phase 1): for every vertex v
 * of the graph, a beam search for x_v seeded at v with ef = k_plus + 1; v is
 * dropped and the next k_plus results form N+(v).
 *   out_nplus   device [n * k_plus] local ids, -1 padded
 */
RNSM_API rnsm_status rnsm_expand(const float *vecs, int64_t n, int32_t dim, const int32_t *adj,
                        int32_t r_in, int32_t k_plus, int32_t metric, int32_t *out_nplus,
                        void *stream);

/*
 * rnsm_reverse_knn -- BuildReverseIndex of Algorithm 2 (Phase 1):
 * R_k(x) = { y : x among the first k entries of N+(y) }, as CSR.
 *   nplus       device [n * k_plus]
 *   out_offs    device [n + 1] int64 offsets (exact)
 *   out_ids     device [n * k] members; each R_k(x) holds exactly its set of
 *               y, listed in ascending order
 */
RNSM_API rnsm_status rnsm_reverse_knn(const int32_t *nplus, int64_t n, int32_t k_plus, int32_t k,
                             int64_t *out_offs, int32_t *out_ids, void *stream);

/*
 * rnsm_select_pivots -- Phase 2 of Algorithm 2 (lazy greedy), on the host.
 * Max-heap on (|R_k(x) \ Covered|, then lower id); a popped x that is
 * covered is skipped, a stale gain is reinserted, otherwise x becomes a pivot
 * with followers F_x = R_k(x) \ Covered and Covered gains {x} u R_k(x).
 *   offs, ids     host CSR of R_k (as rnsm_reverse_knn writes it)
 *   pivot_of      host [n]: pivot of each follower, -1 for pivots
 *   pivots        host [n]: pivots in selection order; *n_pivots their count
 */
RNSM_API rnsm_status rnsm_select_pivots(int64_t n, const int64_t *offs, const int32_t *ids,
                               int32_t *pivot_of, int32_t *pivots, int64_t *n_pivots);

/*
 * rnsm_select_pivots_gpu -- Phase 2 of Algorithm 2 on the device, with the
 * same result as rnsm_select_pivots.  Parallel rounds: every uncovered x whose
 * key (|R_k(x) \ Covered|, then lower id) beats that of every uncovered
 * vertex of N_k(x), R_k(x) and N_k(z) for uncovered z in R_k(x) becomes a
 * pivot with followers R_k(x) \ Covered.  Such local maxima are exactly the
 * vertices the sequential lazy greedy selects with those follower sets.
 *   nplus, k_plus, k   device N+ [n * k_plus]; N_k = its first k columns
 *   offs, ids          device CSR of R_k built from the same N_k
 *   pivot_of           device [n]: pivot of each follower, -1 for pivots
 *   n_pivots, rounds   host outputs (rounds may be NULL)
 */
RNSM_API rnsm_status rnsm_select_pivots_gpu(const int32_t *nplus, int64_t n, int32_t k_plus,
                                            int32_t k, const int64_t *offs, const int32_t *ids,
                                            int32_t *pivot_of, int64_t *n_pivots,
                                            int32_t *rounds, void *stream);

/*
 * rnsm_prune -- heuristic edge selection of UpdateGraph (Section 4.2; the
 * RNG-variant rule of Section 2.2) for a batch of owners over one vector set.
 * For owner v with pool W: drop v, -1 and duplicates; order by (d(v,c), id);
 * keep c unless a kept s has alpha * d(s, c) <= d(v, c) (decided as
 * fmaf(alpha, d(s,c), -d(v,c)) <= 0); stop at R.  With keep_all_if_fit, a
 * pool of at most R distinct candidates is kept whole, in order.
 *   vecs, n, dim      device vector table that owner and pool ids index
 *   owners, nv        device [nv] owner ids
 *   pool, w_len       device [nv * w_len] candidate ids (-1 = none), w_len <= 2048
 *   out               device [nv * R], -1 padded
 */
RNSM_API rnsm_status rnsm_prune(const float *vecs, int64_t n, int32_t dim, const int32_t *owners,
                       int64_t nv, const int32_t *pool, int32_t w_len, int32_t R, float alpha,
                       int32_t metric, int32_t keep_all_if_fit, int32_t prec, int32_t *out,
                       void *stream);

/*
 * rnsm_prune_noalloc -- rnsm_prune (FP32) that allocates no device memory.
 * The paper has no counterpart to this entry point; it exists for callers
 * that cannot let a library allocate: services that give all device memory
 * to their own pool allocator up front and leave no headroom for a
 * library's cudaMalloc, and latency-critical paths that cannot afford the
 * device-wide synchronisation that cudaMalloc and cudaFree may imply.
 * Its scratch (work counters, error word, a list of owners with pools over
 * 64 candidates) is a static device array of 256 B + 4 B per owner for
 * RNSM_PRUNE_NOALLOC_MAX_OWNERS owners (1 MiB), held by every device that
 * loads the library until the process exits.
 *   Arguments, layout and results as rnsm_prune (prec is always FP32).
 *   nv > RNSM_PRUNE_NOALLOC_MAX_OWNERS gives RNSM_EINVAL.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current) and keeps it for the
 * process; make that first call before any stream capture.  A device reset
 * (cudaDeviceReset) reloads the module, so calls after one are invalid.
 * Like every entry point here, the call synchronises `stream` (it reads the
 * validation and error words back to the host) and returns once its outputs
 * are written.  Every call on a device shares the one array (each call
 * clears its counters first): calls that overlap on the GPU, from several
 * host threads or streams, race and must be serialised by the caller.
 */
#define RNSM_PRUNE_NOALLOC_MAX_OWNERS 262144
RNSM_API rnsm_status rnsm_prune_noalloc(const float *vecs, int64_t n, int32_t dim,
                                        const int32_t *owners, int64_t nv, const int32_t *pool,
                                        int32_t w_len, int32_t R, float alpha, int32_t metric,
                                        int32_t keep_all_if_fit, int32_t *out, void *stream);

/*
 * rnsm_reverse_edges -- the target side of UpdateGraph (Section 4.2): target
 * vertices gain cross edges only through the reverse edges of the kept
 * source edges.  Edges (u <- v) are grouped by u with a counting sort
 * (histogram, exclusive scan, scatter); for each u, pool = lists[u] u {v};
 * a pool of at most R distinct entries is kept as is (sorted by (d, id)),
 * a larger one is pruned.
 *   vecs, n, dim      device vector table over all ids
 *   lists             device [n * R] current lists, updated in place
 *   eu, ev, ne        device [ne] edge targets u and sources v
 */
RNSM_API rnsm_status rnsm_reverse_edges(const float *vecs, int64_t n, int32_t dim, int32_t *lists,
                               int32_t R, const int32_t *eu, const int32_t *ev, int64_t ne,
                               float alpha, int32_t metric, void *stream);

/*
 * rnsm_build_segment -- input preparation: the two-stage PG build of
 * Section 2.2 (beam search, occlusion prune, reverse edges) in
 * batch-synchronous rounds.  The entry point is the medoid (the vertex
 * nearest the centroid); vertices are inserted in id order, entry first, a
 * round inserting min(inserted, batch_max) of them against the graph as it
 * stood at the start of the round (seed = entry, ef = L, all L results are
 * candidates).
 *   vecs, n, dim       device vectors
 *   p                  R, L, alpha, metric used
 *   batch_max          round size cap (0 selects n / 64 clamped to [64, 1024])
 *   out_adj            device [n * R] local ids, -1 padded
 *   out_entry          host: the entry vertex
 */
RNSM_API rnsm_status rnsm_build_segment(const float *vecs, int64_t n, int32_t dim, const rnsm_params *p,
                               int64_t batch_max, int32_t *out_adj, int32_t *out_entry,
                               void *stream);

/* Medoid of a vector set: the vertex nearest (native metric) the centroid,
 * ties to the lower id.  Centroid and distances in FP64. */
RNSM_API rnsm_status rnsm_medoid(const float *vecs, int64_t n, int32_t dim, int32_t metric,
                        int32_t *out_entry, void *stream);

/* Message for the calling thread's last non-OK status ("" if none). */
RNSM_API const char *rnsm_last_error(void);

/* Library version string. */
RNSM_API const char *rnsm_version(void);

#ifdef __cplusplus
}
#endif

#endif /* RNSM_H_ */
