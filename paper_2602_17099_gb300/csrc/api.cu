// C ABI of librnsm: validation, workspace, and the orchestration of the
// merge path (Algorithm 2 per plan edge, plan from Algorithm 3).
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
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
    int32_t *scratch_i;      // misc int
};

// Quantized copies of the rows for the tensor-core prune (prec 1 or 2).
struct QuantBufs {
    int32_t prec = 0;
    void *q = nullptr;
    float *scale = nullptr, *err = nullptr, *norm = nullptr;
};

void take_quant(Bump &b, int64_t n, int32_t dim, int32_t prec, QuantBufs &qb) {
    qb.prec = prec;
    if (prec == 0) return;
    qb.q = b.take<char>((size_t)n * dim * (prec == 2 ? 1 : 2));
    qb.scale = b.take<float>(n);
    qb.err = b.take<float>(n);
    qb.norm = b.take<float>(n);
}

void apply_quant(PruneArgs &a, const QuantBufs *qb, unsigned long long *rechecks) {
    a.rechecks = rechecks;
    if (!qb || qb->prec == 0) return;
    a.prec = qb->prec;
    a.qrows = qb->q;
    a.qscale = qb->scale;
    a.qerr = qb->err;
    a.qnorm = qb->norm;
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
    c.scratch_i = b.take<int32_t>(4);
}

rnsm_status ctl_reset(const Ctl &c, cudaStream_t st) {
    CK(cudaMemsetAsync(c.err, 0, sizeof(int32_t), st));
    CK(cudaMemsetAsync(c.stats, 0, 8 * sizeof(unsigned long long), st));
    CK(cudaMemsetAsync(c.rechecks, 0, sizeof(unsigned long long), st));
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

rnsm_status check_vecs(const float *v, int64_t n, int32_t dim) {
    if (!v) return fail(RNSM_EINVAL, "vector pointer is NULL");
    if (n < 1) return fail(RNSM_EINVAL, "n=%lld must be >= 1", (long long)n);
    if (n >= INT32_MAX) return fail(RNSM_EINVAL, "n must be < 2^31");
    if (dim < 4 || (dim & 3)) return fail(RNSM_EINVAL, "dim=%d must be a positive multiple of 4", dim);
    if (!search_dim_supported(dim)) return fail(RNSM_EINVAL, "dim=%d has no search kernel", dim);
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

PruneArgs prune_defaults() {
    PruneArgs a;
    std::memset(&a, 0, sizeof(a));
    return a;
}

rnsm_status run_prune(PruneArgs a, int32_t *work, const Ctl &c, cudaStream_t st) {
    CK(cudaMemsetAsync(work, 0, 2 * sizeof(int32_t), st));
    a.work = work;
    a.work2 = work + 1;
    a.ovf_list = c.ovf;
    a.ovf_count = c.ovf_count;
    CK(launch_prune(a, st));
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
    apply_quant(a, qb, c.rechecks);
    return run_prune(a, c.work + 6, c, st);
}

}  // namespace

void rnsm::set_last_error(const char *msg) { g_err = msg; }

// ======================================================================= ABI

extern "C" {

const char *rnsm_last_error(void) { return g_err.c_str(); }

const char *rnsm_version(void) { return "rnsm-gb300 0.1 (sm_103a)"; }

void rnsm_release_workspace(void) {
    std::lock_guard<std::mutex> lk(g_mu);
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
    TRY(check_vecs(vecs, n, dim));
    if (nv < 0 || (nv > 0 && (!owners || !out)) || w_len < 0 || w_len > 2048 ||
        (w_len > 0 && nv > 0 && !pool))
        return fail(RNSM_EINVAL, "bad owners, pool or output");
    if (R < 1 || R > 64) return fail(RNSM_EINVAL, "R outside [1, 64]");
    if (!(std::isfinite(alpha) && alpha >= 0.f)) return fail(RNSM_EINVAL, "bad alpha");
    if (metric != 0 && metric != 1) return fail(RNSM_EINVAL, "unknown metric");
    if (prec < RNSM_PREC_FP32 || prec > RNSM_PREC_FP8) return fail(RNSM_EINVAL, "unknown precision");
    const int32_t qprec = prune_tc_supported(dim, prec) ? prec : 0;  // else the FP32 kernels
    if (nv == 0) return RNSM_OK;
    Bump b;
    Ctl c;
    QuantBufs qb;
    take_ctl(b, c, nv);
    take_quant(b, n, dim, qprec, qb);
    TRY(ws_acquire(b.off, b));
    take_ctl(b, c, nv);
    take_quant(b, n, dim, qprec, qb);
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
    if (qprec) CK(launch_quantize(tab, n, dim, qprec, qb.q, qb.scale, qb.err, qb.norm, st));
    apply_quant(a, &qb, c.rechecks);
    TRY(run_prune(a, c.work + 8, c, st));
    TRY(check_err_word(c, st));
    return RNSM_OK;
}

rnsm_status rnsm_reverse_edges(const float *vecs, int64_t n, int32_t dim, int32_t *lists,
                               int32_t R, const int32_t *eu, const int32_t *ev, int64_t ne,
                               float alpha, int32_t metric, void *stream) {
    std::lock_guard<std::mutex> lk(g_mu);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    TRY(check_vecs(vecs, n, dim));
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
    TRY(check_vecs(vecs, n, dim));
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

namespace {

struct PairNeeds {
    int64_t ns, nt;
};

struct MergeBufs {
    int32_t *nplus, *rk_keys, *rk_vals, *rk_ids, *rk_cursor;
    int64_t *rk_offs;
    void *rk_scan;
    size_t rk_scan_bytes;
    int32_t *pivots, *followers, *pivot_of, *res, *eu, *ev;
    void *piv_tmp;
    RevBufs rev;
    QuantBufs qb;
};

void carve_merge(Bump &b, const rnsm_params &p, int64_t ns_max, int64_t nt_max, int64_t n_all,
                 int32_t dim, int32_t qprec, Ctl &c, MergeBufs &m) {
    take_ctl(b, c, ns_max > nt_max ? ns_max : nt_max);
    m.nplus = b.take<int32_t>(ns_max * p.k_plus);
    m.rk_keys = b.take<int32_t>(ns_max * p.k_rev);
    m.rk_vals = b.take<int32_t>(ns_max * p.k_rev);
    m.rk_ids = b.take<int32_t>(ns_max * p.k_rev);
    m.rk_cursor = b.take<int32_t>(ns_max);
    m.rk_offs = b.take<int64_t>(ns_max + 1);
    m.rk_scan_bytes = bucket_scan_tmp_bytes(ns_max);
    m.rk_scan = b.take<char>(m.rk_scan_bytes);
    m.pivots = b.take<int32_t>(ns_max);
    m.followers = b.take<int32_t>(ns_max);
    m.pivot_of = b.take<int32_t>(ns_max);
    m.piv_tmp = b.take<char>(pivot_tmp_bytes(ns_max));
    m.res = b.take<int32_t>(ns_max * p.L);
    m.eu = b.take<int32_t>(ns_max * p.R);
    m.ev = b.take<int32_t>(ns_max * p.R);
    take_rev(b, nt_max, ns_max * p.R, m.rev);
    take_quant(b, n_all, dim, qprec, m.qb);
}

// CUDA events at the step boundaries of one plan edge (S1 .. S7).
struct PhaseClock {
    cudaEvent_t ev[9] = {};
    bool ok = true;
    PhaseClock() {
        for (auto &e : ev) ok = ok && cudaEventCreate(&e) == cudaSuccess;
    }
    ~PhaseClock() {
        for (auto &e : ev)
            if (e) cudaEventDestroy(e);
    }
    void mark(int i, cudaStream_t st) {
        if (ok) cudaEventRecord(ev[i], st);
    }
    // after a stream sync: phase_ms[i + shift] += time from mark i to mark i + 1
    void add(double *phase_ms, int lo, int hi, int shift) {
        if (!ok) return;
        for (int i = lo; i < hi; ++i) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, ev[i], ev[i + 1]) == cudaSuccess) phase_ms[i + shift] += ms;
        }
    }
};

struct SrcCache {
    bool done = false;
    int64_t np = 0, nf = 0;
    std::vector<int32_t> pivot_of, pivots, followers;  // host copies (device S3 keeps its own)
    bool on_device = false;
};

}  // namespace

size_t rnsm_workspace_size(const rnsm_segment *segs, int32_t m, const rnsm_params *pin) {
    rnsm_params p;
    if (resolve_params(pin, p) != RNSM_OK || !segs || m < 1) return 0;
    int64_t nmax = 0, nall = 0;
    for (int32_t s = 0; s < m; ++s) {
        nmax = segs[s].n > nmax ? segs[s].n : nmax;
        nall += segs[s].n;
    }
    const int32_t qprec = prune_tc_supported(segs[0].dim, p.prec) ? p.prec : 0;
    Bump b;
    Ctl c;
    MergeBufs mb;
    carve_merge(b, p, nmax, nmax, nall, segs[0].dim, qprec, c, mb);
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
    std::lock_guard<std::mutex> lk(g_mu);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const long long launches0 = launches_so_far();
    double phase_ms[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    int64_t queries[3] = {0, 0, 0};
    PhaseClock clk;
    clk.mark(0, st);
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
    const int32_t qprec = prune_tc_supported(dim, p.prec) ? p.prec : 0;  // else FP32 kernels
    Bump b;
    Ctl c;
    MergeBufs mb;
    carve_merge(b, p, nmax, nmax, off, dim, qprec, c, mb);
    TRY(ws_acquire(b.off, b));
    carve_merge(b, p, nmax, nmax, off, dim, qprec, c, mb);
    TRY(ctl_reset(c, st));
    for (int32_t s = 0; s < m; ++s)
        TRY(validate_on_device(segs[s].vecs, segs[s].n, dim, segs[s].adj, segs[s].r_in, c, st));
    TRY(check_err_word(c, st));
    for (int32_t s = 0; s < m; ++s)
        CK(launch_init_lists(segs[s].adj, segs[s].n, segs[s].r_in, (int32_t)tab.off[s],
                             out_adj + tab.off[s] * p.R, p.R, st));
    if (qprec)  // BF16 / E4M3 copies of every row for the tensor-core prune tiles
        CK(launch_quantize(tab, off, dim, qprec, mb.qb.q, mb.qb.scale, mb.qb.err, mb.qb.norm, st));
    clk.mark(1, st);
    CK(cudaStreamSynchronize(st));
    clk.add(phase_ms, 0, 1, 0);

    std::vector<SrcCache> cache((size_t)m);
    double host_s = 0.0;
    int64_t n_piv = 0, n_fol = 0;
    unsigned long long rev_total = 0;
    const int32_t ks = p.ef_slide < p.L ? p.ef_slide : p.L;
    const bool cm = (p.flags & RNSM_FLAG_CM) != 0;
    std::vector<int64_t> h_offs;
    std::vector<int32_t> h_ids;
    int32_t lists_for = -1;  // source segment whose pivot lists are in the device buffers

    for (const PlanEdge &e : pl) {
        const rnsm_segment &S = segs[e.src], &T = segs[e.dst];
        const int64_t ns = S.n, nt = T.n;
        const int32_t s0 = (int32_t)tab.off[e.src], t0 = (int32_t)tab.off[e.dst];
        SrcCache &sc = cache[e.src];
        clk.mark(0, st);
        clk.mark(1, st);
        clk.mark(2, st);
        bool reuse_later = false;
        for (size_t j = (size_t)(&e - pl.data()) + 1; j < pl.size(); ++j)
            if (pl[j].src == e.src) reuse_later = true;
        if (!sc.done) {
            bool host_lists = true;
            sc.pivot_of.assign((size_t)ns, -1);
            sc.pivots.clear();
            sc.followers.clear();
            if (cm) {
                for (int64_t v = 0; v < ns; ++v) sc.pivots.push_back((int32_t)v);
            } else {
                // S1: neighbour expansion in the source's own graph.
                SearchArgs a = search_defaults();
                a.base = S.vecs;
                a.n_base = ns;
                a.adj = S.adj;
                a.r_in = S.r_in;
                a.dim = dim;
                a.metric = p.metric;
                a.qvecs = S.vecs;
                a.nq = ns;
                a.seed_mode = kSeedSelf;
                a.ef = p.k_plus + 1;
                a.k = p.k_plus;
                a.exclude_self = 1;
                a.out_ids = mb.nplus;
                a.out_stride = p.k_plus;
                a.out_by_qidx = 1;
                a.stats = c.stats;
                TRY(run_search(a, c.work, st));
                queries[0] += ns;
                clk.mark(1, st);
                // S2: reverse kNN inversion (counting sort by x).
                CK(launch_rk_pairs(mb.nplus, ns, p.k_plus, p.k_rev, mb.rk_keys, mb.rk_vals,
                                   c.ecount, st));
                CK(launch_bucket(mb.rk_keys, mb.rk_vals, ns * p.k_rev, c.ecount, ns, 0, mb.rk_offs,
                                 mb.rk_cursor, mb.rk_ids, mb.rk_scan, mb.rk_scan_bytes, st));
                clk.mark(2, st);
                if (p.flags & RNSM_FLAG_HOST_PIVOTS) {
                    // S3: lazy greedy on the host.
                    h_offs.resize((size_t)ns + 1);
                    h_ids.resize((size_t)(ns * p.k_rev));
                    CK(cudaMemcpyAsync(h_offs.data(), mb.rk_offs, sizeof(int64_t) * (ns + 1),
                                       cudaMemcpyDeviceToHost, st));
                    CK(cudaMemcpyAsync(h_ids.data(), mb.rk_ids, sizeof(int32_t) * ns * p.k_rev,
                                       cudaMemcpyDeviceToHost, st));
                    CK(cudaStreamSynchronize(st));
                    const auto h0 = std::chrono::steady_clock::now();
                    select_pivots_host(ns, h_offs.data(), h_ids.data(), sc.pivot_of.data(),
                                       sc.pivots);
                    for (int64_t y = 0; y < ns; ++y)
                        if (sc.pivot_of[y] >= 0) sc.followers.push_back((int32_t)y);
                    host_s += std::chrono::duration<double>(std::chrono::steady_clock::now() - h0)
                                  .count();
                } else {
                    // S3: the same selection in parallel rounds on the device.
                    int64_t np_ = 0, nf_ = 0;
                    CK(select_pivots_device(mb.nplus, ns, p.k_plus, p.k_rev, mb.rk_offs, mb.rk_ids,
                                            mb.pivot_of, mb.pivots, mb.followers, &np_, &nf_,
                                            nullptr, mb.piv_tmp, c.stats + 6, st));
                    sc.np = np_;
                    sc.nf = nf_;
                    host_lists = false;
                    lists_for = e.src;
                    if (reuse_later) {  // keep a host copy: the device lists get overwritten
                        sc.pivot_of.resize((size_t)ns);
                        sc.pivots.resize((size_t)np_);
                        sc.followers.resize((size_t)nf_);
                        CK(cudaMemcpyAsync(sc.pivot_of.data(), mb.pivot_of, sizeof(int32_t) * ns,
                                           cudaMemcpyDeviceToHost, st));
                        if (np_) CK(cudaMemcpyAsync(sc.pivots.data(), mb.pivots,
                                                    sizeof(int32_t) * np_, cudaMemcpyDeviceToHost, st));
                        if (nf_) CK(cudaMemcpyAsync(sc.followers.data(), mb.followers,
                                                    sizeof(int32_t) * nf_, cudaMemcpyDeviceToHost, st));
                        CK(cudaStreamSynchronize(st));
                    }
                }
            }
            if (host_lists) {
                sc.np = (int64_t)sc.pivots.size();
                sc.nf = (int64_t)sc.followers.size();
                lists_for = -1;
            }
            sc.done = true;
        }
        const int64_t np = sc.np, nf = sc.nf;
        n_piv += np;
        n_fol += nf;
        if (lists_for != e.src) {
            if (np) CK(cudaMemcpyAsync(mb.pivots, sc.pivots.data(), sizeof(int32_t) * np,
                                       cudaMemcpyHostToDevice, st));
            if (nf) CK(cudaMemcpyAsync(mb.followers, sc.followers.data(), sizeof(int32_t) * nf,
                                       cudaMemcpyHostToDevice, st));
            CK(cudaMemcpyAsync(mb.pivot_of, sc.pivot_of.data(), sizeof(int32_t) * ns,
                               cudaMemcpyHostToDevice, st));
            lists_for = e.src;
        }
        clk.mark(3, st);
        // S4: naive search of the pivots from the target's default entry.
        {
            SearchArgs a = search_defaults();
            a.base = T.vecs;
            a.n_base = nt;
            a.adj = T.adj;
            a.r_in = T.r_in;
            a.dim = dim;
            a.metric = p.metric;
            a.qvecs = S.vecs;
            a.qidx = mb.pivots;
            a.nq = np;
            a.seed_mode = kSeedConst;
            a.seed_const = T.entry;
            a.ef = p.L;
            a.k = p.L;
            a.out_ids = mb.res;
            a.out_stride = p.L;
            a.out_by_qidx = 1;
            a.stats = c.stats + 2;
            TRY(run_search(a, c.work, st));
            queries[1] += np;
        }
        clk.mark(4, st);
        // S5: local sliding of the followers from their pivot's results.
        if (nf) {
            SearchArgs a = search_defaults();
            a.base = T.vecs;
            a.n_base = nt;
            a.adj = T.adj;
            a.r_in = T.r_in;
            a.dim = dim;
            a.metric = p.metric;
            a.qvecs = S.vecs;
            a.qidx = mb.followers;
            a.nq = nf;
            a.seed_mode = kSeedTable;
            a.seed_tab = mb.res;
            a.seed_stride = p.L;
            a.n_seeds = ks;
            a.seed_row = mb.pivot_of;
            a.ef = p.ef_slide;
            a.k = p.ef_slide;
            a.out_ids = mb.res;
            a.out_stride = p.L;
            a.out_by_qidx = 1;
            a.stats = c.stats + 4;
            TRY(run_search(a, c.work + 3, st));
            queries[2] += nf;
        }
        clk.mark(5, st);
        // S6: source-side UpdateGraph: list(v) + first c_cross results -> prune.
        CK(cudaMemsetAsync(c.ecount, 0, sizeof(unsigned long long), st));
        {
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
            q.listB = mb.res;
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
            apply_quant(q, &mb.qb, c.rechecks);
            TRY(run_prune(q, c.work + 8, c, st));
        }
        clk.mark(6, st);
        // S7: reverse edges into the target (counting sort by u, then prune).
        TRY(reverse_into(tab, dim, p, out_adj, mb.eu, mb.ev, ns * p.R, c.ecount, t0, nt, -1,
                         mb.rev, c, st, &mb.qb));
        clk.mark(7, st);
        unsigned long long ne = 0;
        CK(cudaMemcpyAsync(&ne, c.ecount, sizeof(ne), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        clk.add(phase_ms, 0, 7, 1);  // marks 0..7 bound S1..S7
        rev_total += ne;
    }
    TRY(check_err_word(c, st));
    if (stats) {
        unsigned long long hs[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        CK(cudaMemcpyAsync(hs, c.stats, sizeof(hs), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        stats->ndc = (int64_t)(hs[0] + hs[2] + hs[4]);
        stats->expansions = (int64_t)(hs[1] + hs[3] + hs[5]);
        for (int i = 0; i < 3; ++i) {
            stats->search_ndc[i] = (int64_t)hs[2 * i];
            stats->search_exp[i] = (int64_t)hs[2 * i + 1];
            stats->search_queries[i] = queries[i];
        }
        stats->launches = launches_so_far() - launches0;
        unsigned long long rc = 0;
        CK(cudaMemcpyAsync(&rc, c.rechecks, sizeof(rc), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        stats->rechecks = (int64_t)rc;
        stats->near_ties = 0;
        stats->pivots = n_piv;
        stats->followers = n_fol;
        stats->reverse_edges = (int64_t)rev_total;
        stats->host_pivot_s = host_s;
        stats->wall_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        for (int i = 0; i < 8; ++i) stats->phase_ms[i] = phase_ms[i];
    }
    return RNSM_OK;
}

}  // extern "C"
