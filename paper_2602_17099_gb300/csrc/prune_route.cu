// Routing of a prune call to its kernels, and the autotuner over the prune
// variants (tensor-core tile shapes and the FP32 kernels); host code only.
#include <stdio.h>
#include <stdlib.h>

#include <map>
#include <mutex>

#include "internal.h"

namespace rnsm {

namespace {

// Prune variants.  Every one takes the FP32 prune's decisions (the tensor-core
// tiles re-decide what their bound leaves open), so they differ only in speed:
//   kVarPair: the BF16 / FP8 pair tile (two owners per 128 x 128 tile; L2,
//             d <= 128, pools <= 64);
//   kVarTile: the general tensor-core tile (one owner per 128 x 144 tile; BF16
//             at L2 with the FP32 rows split into two terms, or the library's
//             stored BF16 / E4M3 terms);
//   kVarFp32: the FP32 kernels (register-blocked triangle for pools <= 64);
//   kVarWalk: the FP32 walk over kept rows (pools <= 64, d <= 128).
enum { kVarFp32 = 0, kVarPair = 1, kVarTile = 2, kVarWalk = 3, kVarCount = 4 };

// One variant over a call's owners: its kernel for the pools it takes, the
// general FP32 kernel for the owners whose pools exceed that kernel's capacity.
cudaError_t run_variant(const PruneArgs &a, int var, cudaStream_t st) {
    const bool pair_ok = a.prec != 0 && prune_pair_ok(a.dim, a.prec, a.metric);
    const bool pair = var == kVarPair;
    // BF16 tiles at the pair tile's L2 shapes split the FP32 rows in two terms;
    // every other tile stages the library's stored terms
    const int terms = var != kVarTile ? 0
                      : pair_ok ? (a.prec == 1 ? 2 : 0)
                      : prune_tc_terms(a.dim, a.prec, a.metric);
    const bool tc = var == kVarTile && terms > 0;
    const int cap = pair ? prune_pair_max_pool() : tc ? prune_tc_max_pool() : kPruneSmallMax;
    const bool small_ok = a.ovf_list && a.ovf_count && a.work2 && a.lenA + a.lenB <= cap;
    if (!small_ok) return launch_prune_general(a, nullptr, nullptr, st);
    cudaError_t e = cudaMemsetAsync(a.ovf_count, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    e = pair ? launch_prune_pair(a, st)
        : tc ? launch_prune_tc(a, st, terms)
        : var == kVarWalk ? launch_walk(a, st)
        : launch_small(a, st);
    if (e != cudaSuccess) return e;
    if (a.lenA + a.lenB + (a.csr_offs ? a.csr_max : 0) <= cap) return cudaSuccess;
    // owners whose pools exceeded the first kernel (the count stays on the device)
    PruneArgs b = a;
    b.work = a.work2;
    e = cudaMemsetAsync(b.work, 0, sizeof(int32_t), st);
    if (e != cudaSuccess) return e;
    return launch_prune_general(b, a.ovf_list, a.ovf_count, st);
}

// The variants that apply to a call, the default (the first) included.
int variants_of(const PruneArgs &a, int *out) {
    int n = 0;
    if (a.prec != 0) {
        const bool pair_ok = prune_pair_ok(a.dim, a.prec, a.metric);
        if (pair_ok && a.lenA + a.lenB <= prune_pair_max_pool()) out[n++] = kVarPair;
        const int terms = pair_ok ? (a.prec == 1 ? 2 : 0) : prune_tc_terms(a.dim, a.prec, a.metric);
        const bool stored = terms == 1 ? a.qrows != nullptr : a.qrows && a.qrows_lo;
        if (terms > 0 && ((terms == 2 && a.prec == 1 && a.metric == 0) || stored) &&
            a.lenA + a.lenB <= prune_tc_max_pool())
            out[n++] = kVarTile;
    }
    // FP32 defaults (calls too small to tune): the walk for the source pools, the
    // triangle for reverse-edge pools (on deep-like rows the walk lost there by 40 %)
    const bool walk_ok = a.dim <= kPruneWalkMaxDim && a.lenA + a.lenB <= kPruneSmallMax;
    if (a.csr_offs) {
        out[n++] = kVarFp32;
        if (walk_ok) out[n++] = kVarWalk;
    } else {
        if (walk_ok) out[n++] = kVarWalk;
        out[n++] = kVarFp32;
    }
    return n;
}

// The owners [o0, o1) of a call as a call of their own.
PruneArgs owner_slice(const PruneArgs &a, int64_t o0, int64_t o1) {
    PruneArgs b = a;
    b.n_owners = o1 - o0;
    if (a.owner_ids) b.owner_ids = a.owner_ids + o0;
    else b.owner_base = a.owner_base + (int32_t)o0;
    if (a.listB) b.listB = a.listB + o0 * a.strideB;
    if (a.csr_offs) b.csr_offs = a.csr_offs + o0;
    if (a.out_by_index) b.out = a.out + o0 * a.R;
    return b;
}

// Autotuner over the variants: the first call of a shape (call site,
// precision, dimension, metric, pool length, reverse-edge pools or not) with at least
// kPruneTuneChunks * kPruneTuneMinChunk owners runs as kPruneTuneChunks
// consecutive slices of its owners, the variants taking turns (the order
// rotating every round), each slice timed with CUDA events on the launching
// stream; the variant with the least time per owner is kept for the process.
// A variant's first slice is left out of its time (it may pay the lazy load
// of its kernel's module).  Every owner is pruned once.  Not while the stream
// is being captured, and for reverse-edge pools only on a call with at least
// kPruneTuneMinEntries incoming entries.  RNSM_TUNE_LOG=1 prints each choice
// and its times to stderr, =2 every slice too.
constexpr int kPruneTuneChunks = 12;
constexpr int64_t kPruneTuneMinChunk = 20000;   // owners per slice: short launches are tail-bound
constexpr int64_t kPruneTuneMinEntries = 100000;   // reverse-edge pools: incoming entries
struct PruneKey {
    int prec, dim, metric, len, csr, site;
    bool operator<(const PruneKey &o) const {
        if (site != o.site) return site < o.site;
        if (prec != o.prec) return prec < o.prec;
        if (dim != o.dim) return dim < o.dim;
        if (metric != o.metric) return metric < o.metric;
        if (len != o.len) return len < o.len;
        return csr < o.csr;
    }
};
std::mutex g_ptune_mu;
std::map<PruneKey, int> g_ptuned;

int forced_prune_variant() {
    const char *f = getenv("RNSM_PRUNE_VARIANT");
    return f && f[0] >= '0' && f[0] < '0' + kVarCount ? f[0] - '0' : -1;
}

}  // namespace

cudaError_t launch_prune(const PruneArgs &a, cudaStream_t st, int *variant) {
    int dummy = -1;
    int &ran = variant ? *variant : dummy;
    if (a.n_owners <= 0) return cudaSuccess;
    if (a.R > 64 || a.dim > 1024 || (a.dim & 3)) return cudaErrorInvalidValue;
    int vars[kVarCount];
    const int nv = variants_of(a, vars);
    auto run = [&](const PruneArgs &x, int v) {
        ran = v;
        if ((v == kVarFp32 || v == kVarWalk) && x.prec != 0) {
            PruneArgs y = x;
            y.prec = 0;
            return run_variant(y, v, st);
        }
        return run_variant(x, v, st);
    };
    const int forced = forced_prune_variant();
    if (forced >= 0)
        for (int k = 0; k < nv; ++k)
            if (vars[k] == forced) return run(a, forced);
    if (nv == 1) return run(a, vars[0]);
    const PruneKey key{a.prec, a.dim, a.metric, a.lenA + a.lenB, a.csr_offs != nullptr, a.tune_site};
    {
        std::lock_guard<std::mutex> lk(g_ptune_mu);
        auto it = g_ptuned.find(key);
        if (it != g_ptuned.end()) return run(a, it->second);
    }
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (a.n_owners < kPruneTuneChunks * kPruneTuneMinChunk || !a.work || !a.work2 ||
        cudaStreamIsCapturing(st, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone)
        return run(a, vars[0]);
    if (a.csr_offs) {
        // reverse-edge pools: most owners of an early call may have no entries
        // (the first batches of a graph build); tune only on a call with work
        int64_t ends[2] = {0, 0};
        if (cudaMemcpyAsync(&ends[0], a.csr_offs, sizeof(int64_t), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaMemcpyAsync(&ends[1], a.csr_offs + a.n_owners, sizeof(int64_t), cudaMemcpyDeviceToHost, st) !=
                cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return run(a, vars[0]);
        if (ends[1] - ends[0] < kPruneTuneMinEntries) return run(a, vars[0]);
    }
    double ms_of[kVarCount] = {}, own_of[kVarCount] = {};
    bool seen[kVarCount] = {};
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return run(a, vars[0]);
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return run(a, vars[0]);
    }
    cudaError_t err = cudaSuccess;
    for (int c = 0; c < kPruneTuneChunks && err == cudaSuccess; ++c) {
        const int v = vars[(c + c / nv) % nv];
        const int64_t o0 = a.n_owners * c / kPruneTuneChunks, o1 = a.n_owners * (c + 1) / kPruneTuneChunks;
        err = cudaMemsetAsync(a.work, 0, sizeof(int32_t), st);
        if (err == cudaSuccess) err = cudaMemsetAsync(a.work2, 0, sizeof(int32_t), st);
        if (err == cudaSuccess) err = cudaEventRecord(e0, st);
        if (err == cudaSuccess) err = run(owner_slice(a, o0, o1), v);
        if (err == cudaSuccess) err = cudaEventRecord(e1, st);
        if (err == cudaSuccess) err = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
        if (seen[v]) {
            ms_of[v] += ms;
            own_of[v] += (double)(o1 - o0);
        }
        seen[v] = true;
        const char *lg = getenv("RNSM_TUNE_LOG");
        if (lg && lg[0] == '2')
            fprintf(stderr, "rnsm prune tuner: slice %d variant %d owners %lld..%lld %.3f ms\n", c, v,
                    (long long)o0, (long long)o1, ms);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err != cudaSuccess) return err;
    int best = vars[0];
    for (int k = 1; k < nv; ++k)
        if (ms_of[vars[k]] * own_of[best] < ms_of[best] * own_of[vars[k]]) best = vars[k];
    const char *lg = getenv("RNSM_TUNE_LOG");
    if (lg && (lg[0] == '1' || lg[0] == '2')) {
        fprintf(stderr, "rnsm prune tuner: site %d prec %d dim %d metric %d len %d csr %d owners %lld:",
                key.site, key.prec, key.dim, key.metric, key.len, key.csr, (long long)a.n_owners);
        for (int k = 0; k < nv; ++k)
            fprintf(stderr, " variant %d %.3f ms / %.0f owners;", vars[k], ms_of[vars[k]], own_of[vars[k]]);
        fprintf(stderr, " chose %d\n", best);
    }
    std::lock_guard<std::mutex> lk(g_ptune_mu);
    g_ptuned[key] = best;
    ran = best;
    return cudaSuccess;
}

}  // namespace rnsm
