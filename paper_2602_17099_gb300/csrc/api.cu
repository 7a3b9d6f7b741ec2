// C ABI of librnsm: validation, workspace, and the orchestration of the
// merge path (Algorithm 2 per plan edge, plan from Algorithm 3).
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "host.h"
#include "internal.h"
#include "rnsm.h"

using namespace rnsm;

namespace {

thread_local std::string g_err;

rnsm_status fail(rnsm_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

#define CK(expr)                                                                          \
    do {                                                                                  \
        cudaError_t e_ = (expr);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return fail(RNSM_ECUDA, "%s failed: %s", #expr, cudaGetErrorString(e_));      \
    } while (0)

#define TRY(expr)                                   \
    do {                                            \
        rnsm_status s_ = (expr);                    \
        if (s_ != RNSM_OK) return s_;               \
    } while (0)

// ---------------------------------------------------------------- workspace

constexpr int kMaxDev = 64;
std::mutex g_mu;
struct DevWs {
    void *ptr = nullptr;
    size_t size = 0;
} g_ws[kMaxDev];

// The captured S4..S7 sequence of the last graph-mode call on a device.
struct GraphCache {
    cudaGraphExec_t exec = nullptr;
    cudaStream_t stream = nullptr;   // capture stream (kept for the process)
    std::string key;
    long long launches = 0;
    void reset() {
        if (exec) cudaGraphExecDestroy(exec);
        exec = nullptr;
        key.clear();
    }
};
GraphCache g_graphs[kMaxDev];

int cur_device() {
    int dev = 0;
    cudaGetDevice(&dev);
    return dev >= 0 && dev < kMaxDev ? dev : 0;
}

// Bump allocator over the device workspace (256-byte aligned slices).
struct Bump {
    char *base = nullptr;
    size_t off = 0;
    size_t cap = 0;  // 0 while sizing
    template <class T>
    T *take(size_t count) {
        off = (off + 255) & ~size_t(255);
        T *p = reinterpret_cast<T *>(base ? base + off : nullptr);
        off += count * sizeof(T);
        return p;
    }
};

rnsm_status ws_acquire(size_t bytes, Bump &b) {
    int dev = 0;
    CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDev) return fail(RNSM_EINVAL, "device index %d out of range", dev);
    DevWs &w = g_ws[dev];
    if (w.size < bytes) {
        if (w.ptr) {
            CK(cudaDeviceSynchronize());
            CK(cudaFree(w.ptr));
            w.ptr = nullptr;
            w.size = 0;
        }
        size_t want = bytes + (bytes >> 3) + (1 << 20);
        cudaError_t e = cudaMalloc(&w.ptr, want);
        if (e != cudaSuccess) {
            cudaGetLastError();
            w.ptr = nullptr;
            return fail(RNSM_ENOMEM, "workspace of %zu bytes: %s", want, cudaGetErrorString(e));
        }
        w.size = want;
    }
    b.base = static_cast<char *>(w.ptr);
    b.off = 0;
    b.cap = w.size;
    return RNSM_OK;
}

// Small per-call device state at the head of the workspace.
struct Ctl {
    int32_t *err;
    int32_t *ovf;            // owners passed from the small-pool prune to the general one
    unsigned long long *ovf_count;
    int32_t *work;           // several work counters
    unsigned long long *stats;  // per search slot s: [2s] ndc, [2s+1] expansions
    unsigned long long *ecount;
    unsigned long long *rechecks;  // prune decisions re-decided in FP32
    unsigned long long *tile_tests;  // occlusion tests evaluated by the tensor-core tiles
    unsigned int *tile_err;  // [4] tile error statistics (see rnsm_stats)
    int32_t *scratch_i;      // misc int
    int32_t *kernel_ran = nullptr;  // host [2]: prune variant of the last S6 / S7 call
};

// Quantized copies of the rows for the tensor-core prune (prec 1 or 2).
struct QuantBufs {
    int32_t prec = 0;
    void *q = nullptr;
    void *qlo = nullptr;   // two-term BF16 tiles of inner-product rows: the low terms
    float *scale = nullptr, *err = nullptr, *norm = nullptr;
    int32_t pair_hi_only = 0;   // pair tile: exact hi terms (set by pair_exactness)
};

void take_quant(Bump &b, int64_t n, int32_t dim, int32_t prec, int32_t metric, QuantBufs &qb) {
    qb.prec = prec;
    qb.q = nullptr;
    qb.qlo = nullptr;
    if (prec == 0) return;
    const int terms = prune_tc_terms(dim, prec, metric);
    // L2 two-term tiles and the small-pool pair tiles centre the FP32 rows on
    // each owner; they store nothing
    if ((terms == 2 && metric == RNSM_METRIC_L2) || prune_pair_ok(dim, prec, metric)) return;
    qb.q = b.take<char>((size_t)n * dim * (prec == 2 ? 1 : 2));
    if (terms == 2) qb.qlo = b.take<char>((size_t)n * dim * (prec == 2 ? 1 : 2));
    qb.scale = b.take<float>(n);
    qb.err = b.take<float>(n);
    qb.norm = b.take<float>(n);
}

void apply_quant(PruneArgs &a, const QuantBufs *qb, unsigned long long *rechecks,
                 unsigned int *tile_err = nullptr, unsigned long long *tile_tests = nullptr) {
    a.rechecks = rechecks;
    a.tile_tests = tile_tests;
    if (!qb || qb->prec == 0) return;
    a.tile_err = tile_err;
    a.prec = qb->prec;
    a.qrows = qb->q;
    a.qrows_lo = qb->qlo;
    a.qscale = qb->scale;
    a.qerr = qb->err;
    a.qnorm = qb->norm;
    a.pair_hi_only = qb->pair_hi_only;
}

// The pair tile stages hi terms only when the rows are integers spanning at most
// 256 (checked on the device once per call).
rnsm_status pair_exactness(const SegTable &tab, int32_t dim, int32_t prec, int32_t metric,
                           const Ctl &c, cudaStream_t st, QuantBufs &qb) {
    qb.pair_hi_only = 0;
    if (prec == 0 || !prune_pair_ok(dim, prec, metric)) return RNSM_OK;
    CK(launch_pair_exact_check(tab, dim, c.work + 12, &qb.pair_hi_only, st));
    return RNSM_OK;
}

constexpr int kWorkSlots = 16;

void take_ctl(Bump &b, Ctl &c, int64_t max_owners = 0) {
    c.err = b.take<int32_t>(1);
    c.ovf = max_owners > 0 ? b.take<int32_t>(max_owners) : nullptr;
    c.ovf_count = b.take<unsigned long long>(1);
    c.work = b.take<int32_t>(kWorkSlots);
    c.stats = b.take<unsigned long long>(8);
    c.ecount = b.take<unsigned long long>(1);
    c.rechecks = b.take<unsigned long long>(1);
    c.tile_tests = b.take<unsigned long long>(1);
    c.tile_err = b.take<unsigned int>(4);
    c.scratch_i = b.take<int32_t>(4);
}

rnsm_status ctl_reset(const Ctl &c, cudaStream_t st) {
    CK(cudaMemsetAsync(c.err, 0, sizeof(int32_t), st));
    CK(cudaMemsetAsync(c.stats, 0, 8 * sizeof(unsigned long long), st));
    CK(cudaMemsetAsync(c.rechecks, 0, sizeof(unsigned long long), st));
    CK(cudaMemsetAsync(c.tile_tests, 0, sizeof(unsigned long long), st));
    CK(cudaMemsetAsync(c.tile_err, 0, 4 * sizeof(unsigned int), st));
    return RNSM_OK;
}

rnsm_status check_err_word(const Ctl &c, cudaStream_t st) {
    int32_t err = 0;
    CK(cudaMemcpyAsync(&err, c.err, sizeof(err), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (err & 1) return fail(RNSM_EGRAPH, "adjacency holds a vertex id outside [-1, n)");
    if (err & 2) return fail(RNSM_EGRAPH, "vectors hold a non-finite value");
    if (err & 16) return fail(RNSM_EGRAPH, "a prune pool exceeded 4096 candidates");
    if (err & 32) return fail(RNSM_EGRAPH, "a reverse-kNN row exceeded 4096 entries");
    if (err & 64) return fail(RNSM_ETIMEOUT, "a tensor-core prune tile did not complete in time");
    if (err) return fail(RNSM_ECUDA, "device error word 0x%x", err);
    return RNSM_OK;
}

// ---------------------------------------------------------------- validation

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

rnsm_status resolve_params(const rnsm_params *in, rnsm_params &p) {
    if (!in) return fail(RNSM_EINVAL, "params is NULL");
    p = *in;
    if (p.R < 1 || p.R > 64) return fail(RNSM_EINVAL, "R=%d outside [1, 64]", p.R);
    if (p.L < 1 || p.L > 256) return fail(RNSM_EINVAL, "L=%d outside [1, 256]", p.L);
    if (!(std::isfinite(p.alpha) && p.alpha >= 0.f))
        return fail(RNSM_EINVAL, "alpha must be finite and >= 0");
    if (p.metric != RNSM_METRIC_L2 && p.metric != RNSM_METRIC_IP)
        return fail(RNSM_EINVAL, "unknown metric %d", p.metric);
    if (p.prec < RNSM_PREC_FP32 || p.prec > RNSM_PREC_FP8)
        return fail(RNSM_EINVAL, "unknown precision %d", p.prec);
    if (p.k_rev == 0) p.k_rev = 5;
    if (p.k_plus == 0) p.k_plus = p.k_rev * 2 > 16 ? p.k_rev * 2 : 16;
    if (p.ef_slide == 0) p.ef_slide = (p.L + 1) / 2;
    if (p.c_cross == 0) p.c_cross = p.ef_slide;
    if (p.k_rev < 1 || p.k_plus < p.k_rev || p.k_plus > 255)
        return fail(RNSM_EINVAL, "need 1 <= k_rev <= k_plus <= 255");
    if (p.ef_slide < 1 || p.ef_slide > p.L) return fail(RNSM_EINVAL, "ef_slide outside [1, L]");
    if (p.c_cross < 1 || p.c_cross > p.ef_slide || p.c_cross > p.L)
        return fail(RNSM_EINVAL, "need 1 <= c_cross <= min(L, ef_slide)");
    return RNSM_OK;
}

// need_search: the call runs the beam search, whose kernels exist for a set of dimensions
rnsm_status check_vecs(const float *v, int64_t n, int32_t dim, bool need_search = true) {
    if (!v) return fail(RNSM_EINVAL, "vector pointer is NULL");
    if (n < 1) return fail(RNSM_EINVAL, "n=%lld must be >= 1", (long long)n);
    if (n >= INT32_MAX) return fail(RNSM_EINVAL, "n must be < 2^31");
    if (dim < 4 || (dim & 3)) return fail(RNSM_EINVAL, "dim=%d must be a positive multiple of 4", dim);
    if (need_search && !search_dim_supported(dim))
        return fail(RNSM_EINVAL, "dim=%d has no search kernel", dim);
    if (dim > 1024) return fail(RNSM_EINVAL, "dim=%d above 1024", dim);
    if (!aligned16(v)) return fail(RNSM_EINVAL, "vectors must be 16-byte aligned");
    return RNSM_OK;
}

rnsm_status check_segments(const rnsm_segment *segs, int32_t m, int32_t R) {
    if (!segs || m < 1 || m > kMaxSeg) return fail(RNSM_EINVAL, "need 1 <= m <= %d segments", kMaxSeg);
    int64_t total = 0;
    for (int32_t s = 0; s < m; ++s) {
        const rnsm_segment &g = segs[s];
        TRY(check_vecs(g.vecs, g.n, g.dim));
        if (g.dim != segs[0].dim) return fail(RNSM_EINVAL, "segment %d has dim %d != %d", s, g.dim, segs[0].dim);
        if (g.r_in < 0 || g.r_in > R) return fail(RNSM_EINVAL, "segment %d: r_in=%d outside [0, R]", s, g.r_in);
        if (g.r_in > 0 && !g.adj) return fail(RNSM_EINVAL, "segment %d: adjacency is NULL", s);
        if (g.entry < 0 || g.entry >= g.n) return fail(RNSM_EINVAL, "segment %d: entry %d outside [0, n)", s, g.entry);
        total += g.n;
    }
    if (total >= INT32_MAX) return fail(RNSM_EINVAL, "total vertices must be < 2^31");
    return RNSM_OK;
}

rnsm_status validate_on_device(const float *v, int64_t n, int32_t dim, const int32_t *adj,
                               int32_t r_in, const Ctl &c, cudaStream_t st) {
    CK(launch_validate_vecs(v, n * dim, c.err, st));
    if (adj && r_in > 0) CK(launch_validate_graph(adj, n, r_in, c.err, st));
    return RNSM_OK;
}

SearchArgs search_defaults() {
    SearchArgs a;
    std::memset(&a, 0, sizeof(a));
    return a;
}

rnsm_status run_search(SearchArgs a, int32_t *work, cudaStream_t st) {
    CK(cudaMemsetAsync(work, 0, sizeof(int32_t), st));
    a.work = work;
    CK(launch_search(a, st));
    return RNSM_OK;
}

// A multi-job search as one launch per job (RNSM_SEARCH_PER_JOB=1: the same
// queries and results, for measuring what one launch over every job gains);
// hj: the host copy of the job table, its sentinel included.
rnsm_status run_search_jobs(const SearchArgs &a, int32_t *work, const std::vector<SearchJob> &hj,
                            cudaStream_t st) {
    const char *f = getenv("RNSM_SEARCH_PER_JOB");
    if (!(f && f[0] == '1') || hj.size() < 3) return run_search(a, work, st);
    for (size_t k = 0; k + 1 < hj.size(); ++k) {
        SearchArgs b = a;
        b.q0 = hj[k].q_begin;
        b.nq = hj[k + 1].q_begin - hj[k].q_begin;
        if (b.nq > 0) TRY(run_search(b, work, st));
    }
    return RNSM_OK;
}

PruneArgs prune_defaults() {
    PruneArgs a;
    std::memset(&a, 0, sizeof(a));
    return a;
}

// slot: 0 an S6 call, 1 an S7 call (recorded in c.kernel_ran), -1 neither
rnsm_status run_prune(PruneArgs a, int32_t *work, const Ctl &c, cudaStream_t st, int slot = -1) {
    CK(cudaMemsetAsync(work, 0, 2 * sizeof(int32_t), st));
    a.work = work;
    a.work2 = work + 1;
    a.ovf_list = c.ovf;
    a.ovf_count = c.ovf_count;
    a.tune_site = slot >= 0 && c.kernel_ran ? slot + 1 : 0;   // a merge's S6 / S7, else any
    int ran = -1;
    CK(launch_prune(a, st, &ran));
    if (slot >= 0 && c.kernel_ran) c.kernel_ran[slot] = ran;
    return RNSM_OK;
}

// Groups edges (u <- v) by u and prunes every touched list (UpdateGraph,
// target side).  keys hold u as ids of the table; [key_lo, key_lo + nkeys)
// is the range of possible targets.
struct RevBufs {
    int64_t *offs;
    int32_t *cursor;
    int32_t *ids;
    void *scan_tmp;
    size_t scan_bytes;
};

void take_rev(Bump &b, int64_t nkeys, int64_t cap, RevBufs &r) {
    r.offs = b.take<int64_t>(nkeys + 1);
    r.cursor = b.take<int32_t>(nkeys > 0 ? nkeys : 1);
    r.ids = b.take<int32_t>(cap > 0 ? cap : 1);
    r.scan_bytes = bucket_scan_tmp_bytes(nkeys);
    r.scan_tmp = b.take<char>(r.scan_bytes);
}

rnsm_status reverse_into(const SegTable &tab, int32_t dim, const rnsm_params &p, int32_t *lists,
                         const int32_t *eu, const int32_t *ev, int64_t cap,
                         const unsigned long long *count, int32_t key_lo, int64_t nkeys,
                         int32_t csr_max_bound, const RevBufs &r, const Ctl &c, cudaStream_t st,
                         const QuantBufs *qb = nullptr) {
    CK(launch_bucket(eu, ev, cap, count, nkeys, key_lo, r.offs, r.cursor, r.ids, r.scan_tmp,
                     r.scan_bytes, st));
    int32_t csr_max = csr_max_bound;
    if (csr_max < 0) {
        CK(launch_max_row(r.offs, nkeys, c.scratch_i, st));
        CK(cudaMemcpyAsync(&csr_max, c.scratch_i, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
    }
    PruneArgs a = prune_defaults();
    a.segs = tab;
    a.dim = dim;
    a.metric = p.metric;
    a.alpha = p.alpha;
    a.R = p.R;
    a.keep_all_if_fit = 1;
    a.skip_empty_csr = 1;
    a.n_owners = nkeys;
    a.owner_base = key_lo;
    a.listA = lists;
    a.lenA = p.R;
    a.csr_offs = r.offs;
    a.csr_ids = r.ids;
    a.csr_max = csr_max;
    a.out = lists;
    a.err = c.err;
    apply_quant(a, qb, c.rechecks, c.tile_err, c.tile_tests);
    return run_prune(a, c.work + 6, c, st, 1);
}

}  // namespace

void rnsm::set_last_error(const char *msg) { g_err = msg; }

// ======================================================================= ABI

extern "C" {

const char *rnsm_last_error(void) { return g_err.c_str(); }

const char *rnsm_version(void) { return "rnsm-gb300 0.1 (sm_103a)"; }

void rnsm_release_workspace(void) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_graphs[cur_device()].reset();   // captured launches point into the workspace
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) return;
    if (g_ws[dev].ptr) {
        cudaDeviceSynchronize();
        cudaFree(g_ws[dev].ptr);
    }
    g_ws[dev].ptr = nullptr;
    g_ws[dev].size = 0;
}

rnsm_status mos_plan(int32_t m, const int64_t *sizes, const float *centroids, int32_t D,
                     int32_t degree_bound, int32_t diameter_bound, mos_edge *out,
                     int32_t *n_out) {
    if (m < 1 || !sizes || !n_out) return fail(RNSM_EINVAL, "mos_plan: need m >= 1, sizes, n_out");
    if (centroids && D < 1) return fail(RNSM_EINVAL, "mos_plan: D must be >= 1 with centroids");
    if (degree_bound < 0 || diameter_bound < 0)
        return fail(RNSM_EINVAL, "mos_plan: bounds must be >= 0");
    std::vector<PlanEdge> plan;
    mos_plan_host(m, sizes, centroids, D, degree_bound, diameter_bound, plan);
    if ((int64_t)plan.size() > *n_out || (!out && !plan.empty())) {
        *n_out = (int32_t)plan.size();
        return fail(RNSM_EINVAL, "mos_plan: capacity %d below the %zu plan edges", *n_out,
                    plan.size());
    }
    for (size_t i = 0; i < plan.size(); ++i) {
        out[i].src = plan[i].src;
        out[i].dst = plan[i].dst;
        out[i].cost = plan[i].cost;
    }
    *n_out = (int32_t)plan.size();
    return RNSM_OK;
}

rnsm_status rnsm_select_pivots(int64_t n, const int64_t *offs, const int32_t *ids,
                               int32_t *pivot_of, int32_t *pivots, int64_t *n_pivots) {
    if (n < 1 || !offs || !pivot_of || !pivots || !n_pivots)
        return fail(RNSM_EINVAL, "rnsm_select_pivots: bad arguments");
    if (offs[0] != 0) return fail(RNSM_EINVAL, "rnsm_select_pivots: offs[0] must be 0");
    for (int64_t x = 0; x < n; ++x)
        if (offs[x + 1] < offs[x]) return fail(RNSM_EINVAL, "rnsm_select_pivots: offsets decrease");
    if (offs[n] > 0 && !ids) return fail(RNSM_EINVAL, "rnsm_select_pivots: ids is NULL");
    for (int64_t e = 0; e < offs[n]; ++e)
        if (ids[e] < 0 || ids[e] >= n) return fail(RNSM_EGRAPH, "rnsm_select_pivots: id out of range");
    std::vector<int32_t> piv;
    *n_pivots = select_pivots_host(n, offs, ids, pivot_of, piv);
    std::memcpy(pivots, piv.data(), piv.size() * sizeof(int32_t));
    return RNSM_OK;
}

rnsm_status rnsm_select_pivots_gpu(const int32_t *nplus, int64_t n, int32_t k_plus, int32_t k,
                                   const int64_t *offs, const int32_t *ids, int32_t *pivot_of,
                                   int64_t *n_pivots, int32_t *rounds, void *stream) {
    std::lock_guard<std::mutex> lk(g_mu);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (!nplus || n < 1 || n >= INT32_MAX || !offs || !ids || !pivot_of || !n_pivots)
        return fail(RNSM_EINVAL, "rnsm_select_pivots_gpu: bad arguments");
    if (k < 1 || k > k_plus) return fail(RNSM_EINVAL, "need 1 <= k <= k_plus");
    Bump b;
    Ctl c;
    auto carve = [&](Bump &bb) {
        take_ctl(bb, c);
        int32_t *pv = bb.take<int32_t>(n);
        int32_t *fl = bb.take<int32_t>(n);
        void *tmp = bb.take<char>(pivot_tmp_bytes(n));
        return std::make_tuple(pv, fl, tmp);
    };
    carve(b);
    TRY(ws_acquire(b.off, b));
    int32_t *pv, *fl;
    void *tmp;
    std::tie(pv, fl, tmp) = carve(b);
    TRY(ctl_reset(c, st));
    CK(launch_validate_ids(nplus, n * k_plus, n, 1, c.err, st));
    TRY(check_err_word(c, st));
    int64_t nf = 0;
    CK(select_pivots_device(nplus, n, k_plus, k, offs, ids, pivot_of, pv, fl, n_pivots, &nf,
                            rounds, tmp, c.stats, st));
    return RNSM_OK;
}

rnsm_status rnsm_search(const float *vecs, int64_t n, int32_t dim, const int32_t *adj,
                        int32_t r_in, const float *queries, int64_t nq, const int32_t *seeds,
                        int32_t n_seeds, int32_t ef, int32_t k, int32_t metric,
                        int32_t *out_ids, float *out_dists, int64_t *out_ndc, void *stream) {
    std::lock_guard<std::mutex> lk(g_mu);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    TRY(check_vecs(vecs, n, dim));
    if (r_in < 0 || (r_in > 0 && !adj)) return fail(RNSM_EINVAL, "bad adjacency");
    if (nq < 0 || (nq > 0 && (!queries || !aligned16(queries) || !out_ids)))
        return fail(RNSM_EINVAL, "bad queries or outputs");
    if (n_seeds < 1 || !seeds) return fail(RNSM_EINVAL, "need n_seeds >= 1 seeds per query");
    if (ef < 1 || ef > 256 || k < 1 || k > ef) return fail(RNSM_EINVAL, "need 1 <= k <= ef <= 256");
    if (metric != 0 && metric != 1) return fail(RNSM_EINVAL, "unknown metric");
    if (nq == 0) return RNSM_OK;
    Bump b;
    Ctl c;
    take_ctl(b, c);
    TRY(ws_acquire(b.off, b));
    take_ctl(b, c);
    TRY(ctl_reset(c, st));
    TRY(validate_on_device(vecs, n, dim, adj, r_in, c, st));
    CK(launch_validate_ids(seeds, nq * n_seeds, n, 1, c.err, st));  // -1 or a vertex
    TRY(check_err_word(c, st));
    SearchArgs a = search_defaults();
    a.base = vecs;
    a.n_base = n;
    a.adj = adj;
    a.r_in = r_in;
    a.dim = dim;
    a.metric = metric;
    a.qvecs = queries;
    a.nq = nq;
    a.seed_mode = kSeedTable;
    a.seed_tab = seeds;
    a.seed_stride = n_seeds;
    a.n_seeds = n_seeds;
    a.ef = ef;
    a.k = k;
    a.out_ids = out_ids;
    a.out_stride = k;
    a.out_d = out_dists;
    a.out_ndc = out_ndc;
    a.stats = c.stats;
    TRY(run_search(a, c.work, st));
    TRY(check_err_word(c, st));
    return RNSM_OK;
}

rnsm_status rnsm_expand(const float *vecs, int64_t n, int32_t dim, const int32_t *adj,
                        int32_t r_in, int32_t k_plus, int32_t metric, int32_t *out_nplus,
                        void *stream) {
    std::lock_guard<std::mutex> lk(g_mu);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    TRY(check_vecs(vecs, n, dim));
    if (r_in < 0 || (r_in > 0 && !adj) || !out_nplus) return fail(RNSM_EINVAL, "bad arguments");
    if (k_plus < 1 || k_plus > 255) return fail(RNSM_EINVAL, "k_plus outside [1, 255]");
    if (metric != 0 && metric != 1) return fail(RNSM_EINVAL, "unknown metric");
    Bump b;
    Ctl c;
    take_ctl(b, c);
    TRY(ws_acquire(b.off, b));
    take_ctl(b, c);
    TRY(ctl_reset(c, st));
    TRY(validate_on_device(vecs, n, dim, adj, r_in, c, st));
    TRY(check_err_word(c, st));
    SearchArgs a = search_defaults();
    a.base = vecs;
    a.n_base = n;
    a.adj = adj;
    a.r_in = r_in;
    a.dim = dim;
    a.metric = metric;
    a.qvecs = vecs;
    a.nq = n;
    a.seed_mode = kSeedSelf;
    a.ef = k_plus + 1;
    a.k = k_plus;
    a.exclude_self = 1;
    a.out_ids = out_nplus;
    a.out_stride = k_plus;
    a.out_by_qidx = 1;
    a.stats = c.stats;
    TRY(run_search(a, c.work, st));
    TRY(check_err_word(c, st));
    return RNSM_OK;
}

rnsm_status rnsm_reverse_knn(const int32_t *nplus, int64_t n, int32_t k_plus, int32_t k,
                             int64_t *out_offs, int32_t *out_ids, void *stream) {
    std::lock_guard<std::mutex> lk(g_mu);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (!nplus || n < 1 || n >= INT32_MAX || !out_offs || !out_ids)
        return fail(RNSM_EINVAL, "bad arguments");
    if (k < 1 || k > k_plus) return fail(RNSM_EINVAL, "need 1 <= k <= k_plus");
    Bump b;
    Ctl c;
    RevBufs r;
    take_ctl(b, c);
    int32_t *keys = b.take<int32_t>(n * k), *vals = b.take<int32_t>(n * k);
    take_rev(b, n, 0, r);
    TRY(ws_acquire(b.off, b));
    take_ctl(b, c);
    keys = b.take<int32_t>(n * k);
    vals = b.take<int32_t>(n * k);
    take_rev(b, n, 0, r);
    TRY(ctl_reset(c, st));
    CK(launch_validate_ids(nplus, n * k_plus, n, 1, c.err, st));
    TRY(check_err_word(c, st));
    CK(launch_rk_pairs(nplus, n, k_plus, k, keys, vals, c.ecount, st));
    CK(launch_bucket(keys, vals, n * k, c.ecount, n, 0, out_offs, r.cursor, out_ids, r.scan_tmp,
                     r.scan_bytes, st));
    CK(launch_sort_rows(out_offs, out_ids, n, c.err, st));
    TRY(check_err_word(c, st));
    return RNSM_OK;
}

rnsm_status rnsm_prune(const float *vecs, int64_t n, int32_t dim, const int32_t *owners,
                       int64_t nv, const int32_t *pool, int32_t w_len, int32_t R, float alpha,
                       int32_t metric, int32_t keep_all_if_fit, int32_t prec, int32_t *out,
                       void *stream) {
    std::lock_guard<std::mutex> lk(g_mu);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    TRY(check_vecs(vecs, n, dim, false));
    if (nv < 0 || (nv > 0 && (!owners || !out)) || w_len < 0 || w_len > 2048 ||
        (w_len > 0 && nv > 0 && !pool))
        return fail(RNSM_EINVAL, "bad owners, pool or output");
    if (R < 1 || R > 64) return fail(RNSM_EINVAL, "R outside [1, 64]");
    if (!(std::isfinite(alpha) && alpha >= 0.f)) return fail(RNSM_EINVAL, "bad alpha");
    if (metric != 0 && metric != 1) return fail(RNSM_EINVAL, "unknown metric");
    if (prec < RNSM_PREC_FP32 || prec > RNSM_PREC_FP8) return fail(RNSM_EINVAL, "unknown precision");
    const int32_t qprec = prune_tc_terms(dim, prec) ? prec : 0;  // else the FP32 kernels
    if (nv == 0) return RNSM_OK;
    Bump b;
    Ctl c;
    QuantBufs qb;
    take_ctl(b, c, nv);
    take_quant(b, n, dim, qprec, metric, qb);
    TRY(ws_acquire(b.off, b));
    take_ctl(b, c, nv);
    take_quant(b, n, dim, qprec, metric, qb);
    TRY(ctl_reset(c, st));
    TRY(validate_on_device(vecs, n, dim, nullptr, 0, c, st));
    CK(launch_validate_ids(owners, nv, n, 0, c.err, st));
    if (w_len > 0) CK(launch_validate_ids(pool, nv * w_len, n, 1, c.err, st));
    TRY(check_err_word(c, st));
    SegTable tab;
    std::memset(&tab, 0, sizeof(tab));
    tab.base[0] = vecs;
    tab.off[0] = 0;
    tab.off[1] = n;
    tab.m = 1;
    PruneArgs a = prune_defaults();
    a.segs = tab;
    a.dim = dim;
    a.metric = metric;
    a.alpha = alpha;
    a.R = R;
    a.keep_all_if_fit = keep_all_if_fit;
    a.n_owners = nv;
    a.owner_ids = owners;
    a.listB = pool;
    a.strideB = w_len;
    a.lenB = w_len;
    a.out = out;
    a.out_by_index = 1;
    a.err = c.err;
    if (qb.q) CK(launch_quantize(tab, n, dim, qprec, qb.q, qb.qlo, qb.scale, qb.err, qb.norm, st));
    TRY(pair_exactness(tab, dim, qprec, metric, c, st, qb));
    apply_quant(a, &qb, c.rechecks, nullptr, c.tile_tests);
    TRY(run_prune(a, c.work + 8, c, st));
    TRY(check_err_word(c, st));
    return RNSM_OK;
}

rnsm_status rnsm_reverse_edges(const float *vecs, int64_t n, int32_t dim, int32_t *lists,
                               int32_t R, const int32_t *eu, const int32_t *ev, int64_t ne,
                               float alpha, int32_t metric, void *stream) {
    std::lock_guard<std::mutex> lk(g_mu);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    TRY(check_vecs(vecs, n, dim, false));
    if (!lists || R < 1 || R > 64 || ne < 0 || (ne > 0 && (!eu || !ev)))
        return fail(RNSM_EINVAL, "bad arguments");
    if (!(std::isfinite(alpha) && alpha >= 0.f)) return fail(RNSM_EINVAL, "bad alpha");
    if (metric != 0 && metric != 1) return fail(RNSM_EINVAL, "unknown metric");
    if (ne == 0) return RNSM_OK;
    Bump b;
    Ctl c;
    RevBufs r;
    take_ctl(b, c, n);
    take_rev(b, n, ne, r);
    TRY(ws_acquire(b.off, b));
    take_ctl(b, c, n);
    take_rev(b, n, ne, r);
    TRY(ctl_reset(c, st));
    TRY(validate_on_device(vecs, n, dim, lists, R, c, st));
    CK(launch_validate_ids(eu, ne, n, 0, c.err, st));
    CK(launch_validate_ids(ev, ne, n, 0, c.err, st));
    TRY(check_err_word(c, st));
    SegTable tab;
    std::memset(&tab, 0, sizeof(tab));
    tab.base[0] = vecs;
    tab.off[1] = n;
    tab.m = 1;
    rnsm_params p;
    std::memset(&p, 0, sizeof(p));
    p.R = R;
    p.alpha = alpha;
    p.metric = metric;
    TRY(reverse_into(tab, dim, p, lists, eu, ev, ne, nullptr, 0, n, -1, r, c, st));
    TRY(check_err_word(c, st));
    return RNSM_OK;
}

rnsm_status rnsm_medoid(const float *vecs, int64_t n, int32_t dim, int32_t metric,
                        int32_t *out_entry, void *stream) {
    std::lock_guard<std::mutex> lk(g_mu);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    TRY(check_vecs(vecs, n, dim, false));
    if (!out_entry) return fail(RNSM_EINVAL, "out_entry is NULL");
    Bump b;
    Ctl c;
    take_ctl(b, c);
    const size_t mb = medoid_tmp_bytes(n, dim);
    b.take<char>(mb);
    TRY(ws_acquire(b.off, b));
    take_ctl(b, c);
    double *tmp = reinterpret_cast<double *>(b.take<char>(mb));
    TRY(ctl_reset(c, st));
    CK(launch_medoid(vecs, n, dim, metric, tmp, mb, c.scratch_i, st));
    CK(cudaMemcpyAsync(out_entry, c.scratch_i, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return RNSM_OK;
}

rnsm_status rnsm_build_segment(const float *vecs, int64_t n, int32_t dim, const rnsm_params *pin,
                               int64_t batch_max, int32_t *out_adj, int32_t *out_entry,
                               void *stream) {
    rnsm_params p;
    TRY(resolve_params(pin, p));
    TRY(check_vecs(vecs, n, dim));
    if (!out_adj || !out_entry) return fail(RNSM_EINVAL, "null output");
    if (batch_max < 0) return fail(RNSM_EINVAL, "batch_max must be >= 0");
    if (batch_max == 0) batch_max = n / 64 < 64 ? 64 : (n / 64 > 1024 ? 1024 : n / 64);
    if (batch_max > 4096 - p.R) return fail(RNSM_EINVAL, "batch_max above %d", 4096 - p.R);
    int32_t entry = 0;
    TRY(rnsm_medoid(vecs, n, dim, p.metric, &entry, stream));
    std::lock_guard<std::mutex> lk(g_mu);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    *out_entry = entry;
    Bump b;
    Ctl c;
    RevBufs r;
    const int64_t B = batch_max;
    auto carve = [&](Bump &bb) {
        take_ctl(bb, c, n);
        int32_t *order = bb.take<int32_t>(n);
        int32_t *cand = bb.take<int32_t>(B * p.L);
        int32_t *eu = bb.take<int32_t>(B * p.R);
        int32_t *ev = bb.take<int32_t>(B * p.R);
        take_rev(bb, n, B * p.R, r);
        return std::make_tuple(order, cand, eu, ev);
    };
    carve(b);
    TRY(ws_acquire(b.off, b));
    int32_t *order, *cand, *eu, *ev;
    std::tie(order, cand, eu, ev) = carve(b);
    TRY(ctl_reset(c, st));
    TRY(validate_on_device(vecs, n, dim, nullptr, 0, c, st));
    TRY(check_err_word(c, st));
    {
        std::vector<int32_t> h((size_t)n);
        int64_t k = 0;
        h[k++] = entry;
        for (int64_t i = 0; i < n; ++i)
            if (i != entry) h[k++] = (int32_t)i;
        CK(cudaMemcpyAsync(order, h.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, st));
        CK(launch_fill(out_adj, n * p.R, -1, st));
        CK(cudaStreamSynchronize(st));
    }
    SegTable tab;
    std::memset(&tab, 0, sizeof(tab));
    tab.base[0] = vecs;
    tab.off[1] = n;
    tab.m = 1;
    int64_t inserted = 1;
    while (inserted < n) {
        int64_t bsz = inserted < B ? inserted : B;
        if (bsz > n - inserted) bsz = n - inserted;
        SearchArgs a = search_defaults();
        a.base = vecs;
        a.n_base = n;
        a.adj = out_adj;
        a.r_in = p.R;
        a.dim = dim;
        a.metric = p.metric;
        a.qvecs = vecs;
        a.qidx = order + inserted;
        a.nq = bsz;
        a.seed_mode = kSeedConst;
        a.seed_const = entry;
        a.ef = p.L;
        a.k = p.L;
        a.out_ids = cand;
        a.out_stride = p.L;
        TRY(run_search(a, c.work, st));
        CK(cudaMemsetAsync(c.ecount, 0, sizeof(unsigned long long), st));
        PruneArgs q = prune_defaults();
        q.segs = tab;
        q.dim = dim;
        q.metric = p.metric;
        q.alpha = p.alpha;
        q.R = p.R;
        q.n_owners = bsz;
        q.owner_ids = order + inserted;
        q.listB = cand;
        q.strideB = p.L;
        q.lenB = p.L;
        q.out = out_adj;
        q.emit_lo = 0;
        q.emit_hi = (int32_t)n;
        q.eu = eu;
        q.ev = ev;
        q.ecount = c.ecount;
        q.err = c.err;
        TRY(run_prune(q, c.work + 8, c, st));
        TRY(reverse_into(tab, dim, p, out_adj, eu, ev, bsz * p.R, c.ecount, 0, n, (int32_t)bsz, r,
                         c, st));
        inserted += bsz;
    }
    TRY(check_err_word(c, st));
    return RNSM_OK;
}

// ------------------------------------------------------------------ merge
//
// Execution of a plan (pattern: batched pairs).  Searches read only the
// frozen input graphs, so every search of every plan edge is independent of
// the list updates: the merge runs
//   S1 for every source segment of the plan in one multi-job launch,
//   S2 and S3 per source,
//   S4 for every plan edge of a group in one multi-job launch, then S5 alike,
//   S6 and S7 per plan edge in plan order (they update the lists),
// where a group is a run of consecutive plan edges whose result tables fit
// the result budget (all edges of a plan, unless the segments are huge).
// The results equal those of running Algorithm 2 edge by edge.

namespace {

constexpr size_t kResBudgetBytes = size_t(4) << 30;   // search results of one group

struct MergeBufs {
    int32_t *nplus;                        // [N * k_plus], rows of segment s at off[s]
    int32_t *rk_keys, *rk_vals, *rk_ids, *rk_cursor;
    int64_t *rk_offs;
    void *rk_scan;
    size_t rk_scan_bytes;
    int32_t *pivot_of, *pivots, *followers;   // [N] each, segment s at off[s]
    int32_t *ord, *rank;                      // locality order of each source and positions
    void *piv_tmp;
    int32_t *res;                          // [res_rows * L]
    int32_t *eu, *ev;
    int32_t *upool;                        // union variant: the pools of one source
    SearchJob *jobs1, *jobs4, *jobs5;
    unsigned long long *rev_counts;        // [plan edges] kept cross edges per edge
    RevBufs rev;
    QuantBufs qb;
};

// e_max: the most plan edges of one source (sizes the union variant's pools).
void carve_merge(Bump &b, const rnsm_params &p, int64_t nmax, int64_t n_all, int64_t res_rows,
                 int32_t n_jobs, int32_t dim, int32_t qprec, Ctl &c, MergeBufs &m,
                 int32_t e_max = 1) {
    const bool uni = (p.flags & RNSM_FLAG_UNION) != 0;
    // the union variant prunes the targets of all sources in one pass
    const int64_t nrev = uni ? n_all : nmax;
    take_ctl(b, c, nrev);
    m.nplus = b.take<int32_t>(n_all * p.k_plus);
    m.rk_keys = b.take<int32_t>(nmax * p.k_rev);
    m.rk_vals = b.take<int32_t>(nmax * p.k_rev);
    m.rk_ids = b.take<int32_t>(nmax * p.k_rev);
    m.rk_cursor = b.take<int32_t>(nmax);
    m.rk_offs = b.take<int64_t>(nmax + 1);
    m.rk_scan_bytes = bucket_scan_tmp_bytes(nmax);
    m.rk_scan = b.take<char>(m.rk_scan_bytes);
    m.pivot_of = b.take<int32_t>(n_all);
    m.pivots = b.take<int32_t>(n_all);
    m.followers = b.take<int32_t>(n_all);
    m.ord = b.take<int32_t>(n_all);
    m.rank = b.take<int32_t>(n_all);
    m.piv_tmp = b.take<char>(pivot_tmp_bytes(nmax));
    m.res = b.take<int32_t>(res_rows * p.L);
    m.eu = b.take<int32_t>(nrev * p.R);
    m.ev = b.take<int32_t>(nrev * p.R);
    m.upool = uni ? b.take<int32_t>(nmax * (int64_t)e_max * p.c_cross) : nullptr;
    m.jobs1 = b.take<SearchJob>(n_jobs + 1);
    m.jobs4 = b.take<SearchJob>(n_jobs + 1);
    m.jobs5 = b.take<SearchJob>(n_jobs + 1);
    m.rev_counts = b.take<unsigned long long>(n_jobs + 1);
    take_rev(b, nrev, nrev * p.R, m.rev);
    take_quant(b, n_all, dim, qprec, p.metric, m.qb);
}

// Rows of result table needed by the largest group of the plan.
int64_t plan_res_rows(const rnsm_segment *segs, const std::vector<PlanEdge> &pl, int32_t L) {
    const int64_t budget = (int64_t)(kResBudgetBytes / ((size_t)L * sizeof(int32_t)));
    int64_t best = 0, cur = 0;
    for (const PlanEdge &e : pl) {
        const int64_t ns = segs[e.src].n;
        if (cur > 0 && cur + ns > budget) cur = 0;
        cur += ns;
        best = cur > best ? cur : best;
    }
    return best;
}

// CUDA events around the phases of a merge; elapsed times are summed per
// phase after the final synchronisation.
struct PhaseTimer {
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> spans;
    cudaStream_t st;
    explicit PhaseTimer(cudaStream_t s) : st(s) {}
    ~PhaseTimer() {
        for (auto &sp : spans) {
            cudaEventDestroy(sp.second.first);
            cudaEventDestroy(sp.second.second);
        }
    }
    int begin(int phase) {
        cudaEvent_t a = nullptr, z = nullptr;
        if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&z) != cudaSuccess) {
            if (a) cudaEventDestroy(a);
            cudaGetLastError();
            return -1;
        }
        cudaEventRecord(a, st);
        spans.push_back({phase, {a, z}});
        return (int)spans.size() - 1;
    }
    void end(int idx) {
        if (idx >= 0) cudaEventRecord(spans[(size_t)idx].second.second, st);
    }
    void add(double *phase_ms) const {
        for (const auto &sp : spans) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, sp.second.first, sp.second.second) == cudaSuccess)
                phase_ms[sp.first] += ms;
        }
    }
};

SearchJob make_job(const rnsm_segment &T, const float *qvecs, const int32_t *qidx,
                   int32_t *out_ids, int64_t q_begin) {
    SearchJob j;
    std::memset(&j, 0, sizeof(j));
    j.base = T.vecs;
    j.adj = T.adj;
    j.n_base = T.n;
    j.r_in = T.r_in;
    j.seed_const = T.entry;
    j.qvecs = qvecs;
    j.qidx = qidx;
    j.out_ids = out_ids;
    j.q_begin = q_begin;
    return j;
}

rnsm_status upload_jobs(std::vector<SearchJob> &jobs, int64_t total, SearchJob *dev,
                        cudaStream_t st) {
    SearchJob end;
    std::memset(&end, 0, sizeof(end));
    end.q_begin = total;   // sentinel
    jobs.push_back(end);
    CK(cudaMemcpyAsync(dev, jobs.data(), jobs.size() * sizeof(SearchJob), cudaMemcpyHostToDevice, st));
    return RNSM_OK;
}

rnsm_status resolve_plan(const rnsm_segment *segs, int32_t m, const mos_edge *plan, int32_t n_plan,
                         std::vector<PlanEdge> &pl) {
    if (plan) {
        if (n_plan < 0) return fail(RNSM_EINVAL, "n_plan < 0");
        for (int32_t i = 0; i < n_plan; ++i) {
            if (plan[i].src < 0 || plan[i].src >= m || plan[i].dst < 0 || plan[i].dst >= m ||
                plan[i].src == plan[i].dst)
                return fail(RNSM_EINVAL, "plan edge %d (%d -> %d) is invalid", i, plan[i].src,
                            plan[i].dst);
            pl.push_back({plan[i].src, plan[i].dst, plan[i].cost});
        }
    } else if (m == 2) {
        if (segs[0].n < segs[1].n) pl.push_back({0, 1, 1.0});
        else pl.push_back({1, 0, 1.0});
    } else if (m > 2) {
        return fail(RNSM_EINVAL, "m > 2 needs a plan (mos_plan)");
    }
    return RNSM_OK;
}

// Largest reverse-edge pool a prune accepts (list + incoming); pools above it set
// error bit 16.  Captured launches size the overflow prune for it.
constexpr int32_t kReversePoolBound = 4096;

// Everything the captured launches depend on.
std::string graph_key(const rnsm_segment *segs, int32_t m, const rnsm_params &p,
                      const std::vector<PlanEdge> &pl, const int32_t *out_adj, const char *ws,
                      const std::vector<int64_t> &np, const std::vector<int64_t> &nf, int32_t dim,
                      int32_t qprec) {
    std::string k;
    auto put = [&k](const auto &v) { k.append(reinterpret_cast<const char *>(&v), sizeof(v)); };
    put(m);
    put(dim);
    put(qprec);
    put(p);
    put(out_adj);
    put(ws);
    for (int32_t s = 0; s < m; ++s) {
        put(segs[s].n);
        put(segs[s].dim);
        put(segs[s].r_in);
        put(segs[s].vecs);
        put(segs[s].adj);
        put(segs[s].entry);
        put(np[(size_t)s]);
        put(nf[(size_t)s]);
    }
    for (const PlanEdge &e : pl) {
        put(e.src);
        put(e.dst);
    }
    return k;
}

}  // namespace

size_t rnsm_workspace_size(const rnsm_segment *segs, int32_t m, const rnsm_params *pin) {
    rnsm_params p;
    if (resolve_params(pin, p) != RNSM_OK || !segs || m < 1) return 0;
    int64_t nmax = 0, nall = 0;
    for (int32_t s = 0; s < m; ++s) {
        nmax = segs[s].n > nmax ? segs[s].n : nmax;
        nall += segs[s].n;
    }
    const int32_t qprec = prune_tc_terms(segs[0].dim, p.prec) ? p.prec : 0;
    // a plan of any order: at most m(m-1) edges, results of at most the budget
    const int64_t budget = (int64_t)(kResBudgetBytes / ((size_t)p.L * sizeof(int32_t)));
    int64_t res_rows = nall * (m > 1 ? m - 1 : 1);
    if (res_rows > budget) res_rows = budget > nmax ? budget : nmax;
    Bump b;
    Ctl c;
    MergeBufs mb;
    carve_merge(b, p, nmax, nall, res_rows, m * (m > 1 ? m - 1 : 1), segs[0].dim, qprec, c, mb,
                m > 1 ? m - 1 : 1);
    return b.off;
}

rnsm_status rnsm_merge(const rnsm_segment *segs, int32_t m, const rnsm_params *pin,
                       const mos_edge *plan, int32_t n_plan, int32_t *out_adj, void *stream,
                       rnsm_stats *stats) {
    const auto t0 = std::chrono::steady_clock::now();
    rnsm_params p;
    TRY(resolve_params(pin, p));
    TRY(check_segments(segs, m, p.R));
    if (!out_adj) return fail(RNSM_EINVAL, "out_adj is NULL");
    std::vector<PlanEdge> pl;
    TRY(resolve_plan(segs, m, plan, n_plan, pl));
    std::lock_guard<std::mutex> lk(g_mu);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const long long launches0 = launches_so_far();
    double phase_ms[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    int64_t queries[3] = {0, 0, 0};
    PhaseTimer tm(st);
    const int t_init = tm.begin(0);
    const int32_t dim = segs[0].dim;
    SegTable tab;
    std::memset(&tab, 0, sizeof(tab));
    tab.m = m;
    int64_t off = 0, nmax = 0;
    for (int32_t s = 0; s < m; ++s) {
        tab.base[s] = segs[s].vecs;
        tab.off[s] = off;
        off += segs[s].n;
        nmax = segs[s].n > nmax ? segs[s].n : nmax;
    }
    tab.off[m] = off;
    const int32_t qprec = prune_tc_terms(dim, p.prec) ? p.prec : 0;  // else FP32 kernels
    const int64_t res_rows = plan_res_rows(segs, pl, p.L);
    const int32_t n_jobs = (int32_t)pl.size() > m ? (int32_t)pl.size() : m;
    int32_t e_max = 1;
    {
        std::vector<int32_t> ne((size_t)m, 0);
        for (const PlanEdge &e : pl) e_max = std::max(e_max, ++ne[(size_t)e.src]);
    }
    const bool uni = (p.flags & RNSM_FLAG_UNION) != 0;
    if (uni && (p.flags & RNSM_FLAG_GRAPH))
        return fail(RNSM_EINVAL, "RNSM_FLAG_UNION does not combine with RNSM_FLAG_GRAPH");
    if (uni && res_rows < [&] { int64_t t = 0; for (const PlanEdge &e : pl) t += segs[e.src].n; return t; }())
        return fail(RNSM_EINVAL, "RNSM_FLAG_UNION needs the plan's search results in one group");
    Bump b;
    Ctl c;
    MergeBufs mb;
    carve_merge(b, p, nmax, off, res_rows, n_jobs, dim, qprec, c, mb, e_max);
    TRY(ws_acquire(b.off, b));
    carve_merge(b, p, nmax, off, res_rows, n_jobs, dim, qprec, c, mb, e_max);
    int32_t kernel_ran[2] = {-1, -1};
    c.kernel_ran = kernel_ran;
    TRY(ctl_reset(c, st));
    for (int32_t s = 0; s < m; ++s)
        TRY(validate_on_device(segs[s].vecs, segs[s].n, dim, segs[s].adj, segs[s].r_in, c, st));
    TRY(check_err_word(c, st));
    for (int32_t s = 0; s < m; ++s)
        CK(launch_init_lists(segs[s].adj, segs[s].n, segs[s].r_in, (int32_t)tab.off[s],
                             out_adj + tab.off[s] * p.R, p.R, st));
    if (mb.qb.q)  // BF16 / E4M3 copies of every row for the one-term tensor-core tiles
        CK(launch_quantize(tab, off, dim, qprec, mb.qb.q, mb.qb.qlo, mb.qb.scale, mb.qb.err,
                           mb.qb.norm, st));
    // (a captured graph keeps its launch arguments: the general pair tile there)
    mb.qb.pair_hi_only = 0;
    if (!(p.flags & RNSM_FLAG_GRAPH)) TRY(pair_exactness(tab, dim, qprec, p.metric, c, st, mb.qb));
    tm.end(t_init);

    const int32_t ks = p.ef_slide < p.L ? p.ef_slide : p.L;
    const bool cm = (p.flags & RNSM_FLAG_CM) != 0;
    std::vector<int32_t> srcs;            // source segments in order of first use
    std::vector<char> is_src((size_t)m, 0);
    for (const PlanEdge &e : pl)
        if (!is_src[(size_t)e.src]) {
            is_src[(size_t)e.src] = 1;
            srcs.push_back(e.src);
        }
    std::vector<int64_t> np((size_t)m, 0), nf((size_t)m, 0);
    double host_s = 0.0;
    int64_t n_piv = 0, n_fol = 0;
    unsigned long long rev_total = 0;

    if (cm) {
        // CM: every source vertex is a pivot (naive search), no followers
        for (int32_t s : srcs) {
            std::vector<int32_t> iota((size_t)segs[s].n);
            for (int64_t v = 0; v < segs[s].n; ++v) iota[(size_t)v] = (int32_t)v;
            CK(cudaMemcpyAsync(mb.pivots + tab.off[s], iota.data(), sizeof(int32_t) * iota.size(),
                               cudaMemcpyHostToDevice, st));
            CK(cudaStreamSynchronize(st));
            np[(size_t)s] = segs[s].n;
        }
    } else if (!srcs.empty()) {
        // S1: neighbour expansion of every source in its own graph, one launch,
        // queries in locality order
        const int t1 = tm.begin(1);
        std::vector<SearchJob> jobs;
        int64_t total = 0;
        for (int32_t s : srcs) {
            CK(launch_locality_order(segs[s].vecs, segs[s].n, dim, mb.rk_keys, mb.rk_vals,
                                     mb.rk_offs, mb.rk_cursor, mb.rk_scan, mb.rk_scan_bytes,
                                     mb.ord + tab.off[s], mb.rank + tab.off[s], st));
            jobs.push_back(make_job(segs[s], segs[s].vecs, mb.ord + tab.off[s],
                                    mb.nplus + tab.off[s] * p.k_plus, total));
            total += segs[s].n;
        }
        TRY(upload_jobs(jobs, total, mb.jobs1, st));
        SearchArgs a = search_defaults();
        a.dim = dim;
        a.metric = p.metric;
        a.nq = total;
        a.seed_mode = kSeedSelf;
        a.ef = p.k_plus + 1;
        a.k = p.k_plus;
        a.exclude_self = 1;
        a.out_stride = p.k_plus;
        a.out_by_qidx = 1;
        a.stats = c.stats;
        a.jobs = mb.jobs1;
        a.n_jobs = (int32_t)srcs.size();
        TRY(run_search_jobs(a, c.work, jobs, st));
        queries[0] += total;
        tm.end(t1);
        // S2 (reverse kNN inversion) and S3 (pivots) per source
        for (int32_t s : srcs) {
            const int64_t ns = segs[s].n;
            const int32_t *nplus = mb.nplus + tab.off[s] * p.k_plus;
            int32_t *pivot_of = mb.pivot_of + tab.off[s];
            int32_t *pivots = mb.pivots + tab.off[s];
            int32_t *followers = mb.followers + tab.off[s];
            const int t2 = tm.begin(2);
            CK(launch_rk_pairs(nplus, ns, p.k_plus, p.k_rev, mb.rk_keys, mb.rk_vals, c.ecount, st));
            CK(launch_bucket(mb.rk_keys, mb.rk_vals, ns * p.k_rev, c.ecount, ns, 0, mb.rk_offs,
                             mb.rk_cursor, mb.rk_ids, mb.rk_scan, mb.rk_scan_bytes, st));
            tm.end(t2);
            const int t3 = tm.begin(3);
            if (p.flags & RNSM_FLAG_HOST_PIVOTS) {
                // S3: lazy greedy on the host
                std::vector<int64_t> h_offs((size_t)ns + 1);
                std::vector<int32_t> h_ids((size_t)(ns * p.k_rev)), h_pof((size_t)ns, -1), h_piv, h_fol;
                CK(cudaMemcpyAsync(h_offs.data(), mb.rk_offs, sizeof(int64_t) * (ns + 1),
                                   cudaMemcpyDeviceToHost, st));
                CK(cudaMemcpyAsync(h_ids.data(), mb.rk_ids, sizeof(int32_t) * ns * p.k_rev,
                                   cudaMemcpyDeviceToHost, st));
                CK(cudaStreamSynchronize(st));
                const auto h0 = std::chrono::steady_clock::now();
                select_pivots_host(ns, h_offs.data(), h_ids.data(), h_pof.data(), h_piv);
                for (int64_t y = 0; y < ns; ++y)
                    if (h_pof[(size_t)y] >= 0) h_fol.push_back((int32_t)y);
                host_s += std::chrono::duration<double>(std::chrono::steady_clock::now() - h0).count();
                np[(size_t)s] = (int64_t)h_piv.size();
                nf[(size_t)s] = (int64_t)h_fol.size();
                if (!h_piv.empty())
                    CK(cudaMemcpyAsync(pivots, h_piv.data(), sizeof(int32_t) * h_piv.size(),
                                       cudaMemcpyHostToDevice, st));
                if (!h_fol.empty())
                    CK(cudaMemcpyAsync(followers, h_fol.data(), sizeof(int32_t) * h_fol.size(),
                                       cudaMemcpyHostToDevice, st));
                CK(cudaMemcpyAsync(pivot_of, h_pof.data(), sizeof(int32_t) * ns,
                                   cudaMemcpyHostToDevice, st));
                CK(cudaStreamSynchronize(st));
            } else {
                // S3: the same selection in parallel rounds on the device
                int64_t np_ = 0, nf_ = 0;
                CK(select_pivots_device(nplus, ns, p.k_plus, p.k_rev, mb.rk_offs, mb.rk_ids,
                                        pivot_of, pivots, followers, &np_, &nf_, nullptr,
                                        mb.piv_tmp, c.stats + 6, st));
                np[(size_t)s] = np_;
                nf[(size_t)s] = nf_;
            }
            // schedule of S4 and S5: pivots in locality order, each pivot's followers
            // (which start from the same seeds) side by side
            CK(order_search_lists(mb.rank + tab.off[s], pivot_of, pivots, np[(size_t)s], followers,
                                  nf[(size_t)s], ns, mb.rk_keys, mb.rk_vals, mb.rk_offs,
                                  mb.rk_cursor, mb.rk_scan, mb.rk_scan_bytes, st));
            tm.end(t3);
        }
    }

    // S4 .. S7 over groups of consecutive plan edges
    const int64_t budget = (int64_t)(kResBudgetBytes / ((size_t)p.L * sizeof(int32_t)));
    std::vector<std::pair<size_t, size_t>> groups;
    std::vector<int64_t> res_off(pl.size(), 0);
    for (size_t g0 = 0; g0 < pl.size();) {
        size_t g1 = g0;
        int64_t rows = 0;
        while (g1 < pl.size() && (g1 == g0 || rows + segs[pl[g1].src].n <= budget)) {
            res_off[g1] = rows;
            rows += segs[pl[g1].src].n;
            ++g1;
        }
        groups.push_back({g0, g1});
        g0 = g1;
    }
    // the job tables of a group (host side; uploaded before its launches)
    auto jobs_of = [&](size_t g0, size_t g1, bool followers, int64_t &total) {
        std::vector<SearchJob> jobs;
        total = 0;
        for (size_t e = g0; e < g1; ++e) {
            const int32_t sv = pl[e].src;
            int32_t *res = mb.res + res_off[e] * p.L;
            SearchJob j = make_job(segs[pl[e].dst], segs[sv].vecs,
                                   (followers ? mb.followers : mb.pivots) + tab.off[sv], res, total);
            if (followers) {
                j.seed_tab = res;
                j.seed_row = mb.pivot_of + tab.off[sv];
            }
            jobs.push_back(j);
            total += followers ? nf[(size_t)sv] : np[(size_t)sv];
        }
        return jobs;
    };
    // enqueues S4, S5 and the per-edge S6 / S7 of a group; no host synchronisation
    // when `graph` (the reverse pools are then sized by their static bound)
    auto enqueue_group = [&](size_t gi, bool graph, int64_t tot4, int64_t tot5,
                             const std::vector<SearchJob> &hj4, const std::vector<SearchJob> &hj5,
                             cudaStream_t es) -> rnsm_status {
        const size_t g0 = groups[gi].first, g1 = groups[gi].second;
        int span = graph ? -1 : tm.begin(4);
        {   // S4: naive search of the pivots of every edge of the group, one launch
            SearchArgs a = search_defaults();
            a.dim = dim;
            a.metric = p.metric;
            a.nq = tot4;
            a.seed_mode = kSeedConst;
            a.ef = p.L;
            a.k = p.L;
            a.out_stride = p.L;
            a.out_by_qidx = 1;
            a.stats = c.stats + 2;
            a.jobs = mb.jobs4;
            a.n_jobs = (int32_t)(g1 - g0);
            TRY(run_search_jobs(a, c.work, hj4, es));
        }
        tm.end(span);
        span = graph ? -1 : tm.begin(5);
        if (tot5 > 0) {   // S5: local sliding of the followers of every edge, one launch
            SearchArgs a = search_defaults();
            a.dim = dim;
            a.metric = p.metric;
            a.nq = tot5;
            a.seed_mode = kSeedTable;
            a.seed_stride = p.L;
            a.n_seeds = ks;
            a.ef = p.ef_slide;
            a.k = p.ef_slide;
            a.out_stride = p.L;
            a.out_by_qidx = 1;
            a.stats = c.stats + 4;
            a.jobs = mb.jobs5;
            a.n_jobs = (int32_t)(g1 - g0);
            TRY(run_search_jobs(a, c.work + 3, hj5, es));
        }
        tm.end(span);
        if (uni) {
            // one prune per source vertex over its union pool, sources in order of
            // their first plan edge; then the kept cross edges of every source and
            // one reverse-edge pass over all ids
            span = graph ? -1 : tm.begin(6);
            UnionMasks mk;
            std::memset(&mk, 0, sizeof(mk));
            for (size_t e = g0; e < g1; ++e) mk.tmask[pl[e].src] |= 1ull << pl[e].dst;
            std::vector<char> done((size_t)m, 0);
            for (size_t e0 = g0; e0 < g1; ++e0) {
                const int32_t sv = pl[e0].src;
                if (done[(size_t)sv]) continue;
                done[(size_t)sv] = 1;
                UnionEdges ue;
                std::memset(&ue, 0, sizeof(ue));
                for (size_t e = e0; e < g1; ++e)
                    if (pl[e].src == sv) {
                        ue.res[ue.n] = mb.res + res_off[e] * p.L;
                        ue.t0[ue.n] = (int32_t)tab.off[pl[e].dst];
                        ++ue.n;
                    }
                const int64_t ns = segs[sv].n;
                CK(launch_union_pool(ue, ns, p.L, p.c_cross, mb.upool, es));
                PruneArgs q = prune_defaults();
                q.segs = tab;
                q.dim = dim;
                q.metric = p.metric;
                q.alpha = p.alpha;
                q.R = p.R;
                q.n_owners = ns;
                q.owner_base = (int32_t)tab.off[sv];
                q.listA = out_adj;
                q.lenA = p.R;
                q.listB = mb.upool;
                q.strideB = ue.n * p.c_cross;
                q.lenB = ue.n * p.c_cross;
                q.offB = 0;
                q.out = out_adj;
                q.err = c.err;
                apply_quant(q, &mb.qb, c.rechecks, c.tile_err, c.tile_tests);
                TRY(run_prune(q, c.work + 8, c, es, 0));
            }
            tm.end(span);
            span = graph ? -1 : tm.begin(7);
            CK(cudaMemsetAsync(c.ecount, 0, sizeof(unsigned long long), es));
            CK(launch_emit_cross(out_adj, p.R, tab, mk, mb.eu, mb.ev, c.ecount, es));
            TRY(reverse_into(tab, dim, p, out_adj, mb.eu, mb.ev, tab.off[m] * p.R, c.ecount, 0,
                             tab.off[m], -1, mb.rev, c, es, &mb.qb));
            CK(cudaMemsetAsync(mb.rev_counts + g0, 0, sizeof(unsigned long long) * (g1 - g0), es));
            CK(cudaMemcpyAsync(mb.rev_counts + g0, c.ecount, sizeof(unsigned long long),
                               cudaMemcpyDeviceToDevice, es));
            tm.end(span);
            return RNSM_OK;
        }
        for (size_t e = g0; e < g1; ++e) {   // S6 and S7 per edge, in plan order
            const PlanEdge &E = pl[e];
            const int64_t ns = segs[E.src].n, nt = segs[E.dst].n;
            const int32_t s0 = (int32_t)tab.off[E.src], t0 = (int32_t)tab.off[E.dst];
            span = graph ? -1 : tm.begin(6);
            CK(cudaMemsetAsync(c.ecount, 0, sizeof(unsigned long long), es));
            PruneArgs q = prune_defaults();
            q.segs = tab;
            q.dim = dim;
            q.metric = p.metric;
            q.alpha = p.alpha;
            q.R = p.R;
            q.n_owners = ns;
            q.owner_base = s0;
            q.listA = out_adj;
            q.lenA = p.R;
            q.listB = mb.res + res_off[e] * p.L;
            q.strideB = p.L;
            q.lenB = p.c_cross;
            q.offB = t0;
            q.out = out_adj;
            q.emit_lo = t0;
            q.emit_hi = t0 + (int32_t)nt;
            q.eu = mb.eu;
            q.ev = mb.ev;
            q.ecount = c.ecount;
            q.err = c.err;
            apply_quant(q, &mb.qb, c.rechecks, c.tile_err, c.tile_tests);
            TRY(run_prune(q, c.work + 8, c, es, 0));
            tm.end(span);
            span = graph ? -1 : tm.begin(7);
            TRY(reverse_into(tab, dim, p, out_adj, mb.eu, mb.ev, ns * p.R, c.ecount, t0, nt,
                             graph ? kReversePoolBound - p.R : -1, mb.rev, c, es, &mb.qb));
            CK(cudaMemcpyAsync(mb.rev_counts + e, c.ecount, sizeof(unsigned long long),
                               cudaMemcpyDeviceToDevice, es));
            tm.end(span);
        }
        return RNSM_OK;
    };
    for (size_t gi = 0; gi < groups.size(); ++gi) {
        int64_t tot4 = 0, tot5 = 0;
        std::vector<SearchJob> j4 = jobs_of(groups[gi].first, groups[gi].second, false, tot4);
        std::vector<SearchJob> j5 = jobs_of(groups[gi].first, groups[gi].second, true, tot5);
        // capture only what replays unchanged: one group, no autotuning inside
        const bool want_graph = (p.flags & RNSM_FLAG_GRAPH) && !uni && groups.size() == 1 &&
                                !search_would_tune(dim, p.L, kSeedConst, tot4) &&
                                !search_would_tune(dim, p.ef_slide, kSeedTable, tot5);
        TRY(upload_jobs(j4, tot4, mb.jobs4, st));
        TRY(upload_jobs(j5, tot5, mb.jobs5, st));
        for (size_t e = groups[gi].first; e < groups[gi].second; ++e) {
            n_piv += np[(size_t)pl[e].src];
            n_fol += nf[(size_t)pl[e].src];
        }
        queries[1] += tot4;
        queries[2] += tot5;
        if (!want_graph) {
            TRY(enqueue_group(gi, false, tot4, tot5, j4, j5, st));
            continue;
        }
        // graph mode: capture once, replay while the key matches
        std::string key = graph_key(segs, m, p, pl, out_adj, b.base, np, nf, dim, qprec);
        GraphCache &gc = g_graphs[cur_device()];
        const bool replay = gc.exec && gc.key == key;
        if (!replay) {
            gc.reset();
            const long long l0 = launches_so_far();
            // capture on the library's own stream (the legacy default stream cannot be
            // captured); the graph is launched on the caller's stream below
            if (!gc.stream) CK(cudaStreamCreateWithFlags(&gc.stream, cudaStreamNonBlocking));
            CK(cudaStreamBeginCapture(gc.stream, cudaStreamCaptureModeRelaxed));
            const rnsm_status rs = enqueue_group(gi, true, tot4, tot5, j4, j5, gc.stream);
            cudaGraph_t graph = nullptr;
            const cudaError_t ce = cudaStreamEndCapture(gc.stream, &graph);
            if (rs != RNSM_OK) {
                if (graph) cudaGraphDestroy(graph);
                return rs;
            }
            CK(ce);
            const cudaError_t ie = cudaGraphInstantiate(&gc.exec, graph, 0);
            cudaGraphDestroy(graph);
            CK(ie);
            gc.key = key;
            gc.launches = launches_so_far() - l0;   // kernels one replay launches
        } else {
            note_launches((int)gc.launches);
        }
        const int span = tm.begin(4);
        CK(cudaGraphLaunch(gc.exec, st));
        tm.end(span);
    }
    {
        std::vector<unsigned long long> rc(pl.size(), 0ull);
        if (!pl.empty())
            CK(cudaMemcpyAsync(rc.data(), mb.rev_counts, sizeof(unsigned long long) * pl.size(),
                               cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        for (unsigned long long v : rc) rev_total += v;
    }
    TRY(check_err_word(c, st));
    if (stats) {
        unsigned long long hs[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        CK(cudaMemcpyAsync(hs, c.stats, sizeof(hs), cudaMemcpyDeviceToHost, st));
        unsigned long long rc = 0;
        unsigned int te[4] = {0, 0, 0, 0};
        CK(cudaMemcpyAsync(&rc, c.rechecks, sizeof(rc), cudaMemcpyDeviceToHost, st));
        unsigned long long tt = 0;
        CK(cudaMemcpyAsync(&tt, c.tile_tests, sizeof(tt), cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(te, c.tile_err, sizeof(te), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        for (int i = 0; i < 3; ++i) {
            float f;
            std::memcpy(&f, &te[i], sizeof(f));
            stats->tile_error[i] = f;
        }
        stats->tile_error[3] = te[3];
        stats->ndc = (int64_t)(hs[0] + hs[2] + hs[4]);
        stats->expansions = (int64_t)(hs[1] + hs[3] + hs[5]);
        for (int i = 0; i < 3; ++i) {
            stats->search_ndc[i] = (int64_t)hs[2 * i];
            stats->search_exp[i] = (int64_t)hs[2 * i + 1];
            stats->search_queries[i] = queries[i];
        }
        stats->launches = launches_so_far() - launches0;
        stats->rechecks = (int64_t)rc;
        stats->tile_tests = (int64_t)tt;
        stats->prune_kernel[0] = kernel_ran[0];
        stats->prune_kernel[1] = kernel_ran[1];
        stats->pivots = n_piv;
        stats->followers = n_fol;
        stats->reverse_edges = (int64_t)rev_total;
        stats->host_pivot_s = host_s;
        tm.add(phase_ms);
        stats->wall_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        for (int i = 0; i < 8; ++i) stats->phase_ms[i] = phase_ms[i];
    }
    return RNSM_OK;
}

}  // extern "C"
