// K1: batched AKNN beam search (Algorithm 1, Section 2.2), one warp per query.
//
// Per warp, in shared memory: the candidate set C as a (distance, id) array
// sorted lexicographically and double buffered (the expanded flag rides in
// bit 31 of the id), an open-addressing visited hash, and staging for the
// distances of the current neighbourhood.  Neighbour rows are gathered with
// 128-bit loads: a group of G lanes covers one row (lane s of the group reads
// float4 s, s+G, ...), 32/G rows per step, U steps in flight.
//
// Semantics match Algorithm 1 exactly: repeatedly expand the nearest
// unexpanded entry, evaluate every neighbour not evaluated before, keep the
// best ef by (distance, id).  Inserting a whole neighbourhood and truncating
// to ef leaves the same set as inserting one neighbour at a time.  The hash
// is exact until a probe sequence runs out; from then on it is lossy, which
// cannot change the result because an evaluated vertex outside C is worse
// than the worst entry of C (and that bound only tightens) while vertices
// inside C are deduplicated by id before insertion.
#include <float.h>
#include <stdlib.h>

#include <map>
#include <mutex>
#include <utility>

#include "search_impl.cuh"

namespace rnsm {

namespace {

cudaError_t launch_dim_any(const SearchArgs &a, int var, cudaStream_t st) {
    return a.jobs ? launch_search_jobs(a, var, st) : launch_dim<false>(a, var, st);
}

// The queries [q0, q1) of a launch as a launch of their own.
SearchArgs subrange(const SearchArgs &a, int64_t q0, int64_t q1) {
    SearchArgs b = a;
    b.q0 = a.q0 + q0;
    b.nq = q1 - q0;
    return b;
}

// Autotuner: the first launch of a (dim, beam, seed mode) shape with at least
// kTuneChunks * kTuneMinChunk queries runs as kTuneChunks consecutive chunks
// spread over its whole query list, the variants taking turns (the order
// rotating every round), each chunk timed with CUDA events on the launching
// stream and its distance computations counted.  The variant with the least
// time per distance computation is kept for later launches of that shape.
// Every query runs once, with final results (all variants compute the same
// beams); normalising by the distance count makes chunks of different
// difficulty comparable, and spreading the chunks over the list keeps the
// comparison representative when the queries come in locality order.
constexpr int kTuneChunks = 4 * kVariants;
constexpr int64_t kTuneMinChunk = 4000;
struct TuneKey {
    int dim, efmax, seed_mode;
    bool operator<(const TuneKey &o) const {
        return dim != o.dim ? dim < o.dim : efmax != o.efmax ? efmax < o.efmax : seed_mode < o.seed_mode;
    }
};
std::mutex g_tune_mu;
std::map<TuneKey, int> g_tuned;

int efmax_of(int ef) { return ef <= 32 ? 32 : ef <= 64 ? 64 : ef <= 128 ? 128 : 256; }

int forced_variant() {
    const char *force = getenv("RNSM_SEARCH_VARIANT");
    return force && force[0] >= '0' && force[0] < '0' + kVariants ? force[0] - '0' : -1;
}

}  // namespace

bool search_would_tune(int dim, int ef, int seed_mode, int64_t nq) {
    if (forced_variant() >= 0 || nq < kTuneChunks * kTuneMinChunk) return false;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    return g_tuned.find({dim, efmax_of(ef), seed_mode}) == g_tuned.end();
}

cudaError_t launch_search(const SearchArgs &a, cudaStream_t st) {
    if (a.nq <= 0) return cudaSuccess;
    if (!search_dim_supported(a.dim)) return cudaErrorInvalidValue;
    const int forced = forced_variant();
    if (forced >= 0) return launch_dim_any(a, forced, st);
    const TuneKey key{a.dim, efmax_of(a.ef), a.seed_mode};
    int var = -1;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tuned.find(key);
        if (it != g_tuned.end()) var = it->second;
    }
    if (var >= 0 || a.nq < kTuneChunks * kTuneMinChunk) return launch_dim_any(a, var >= 0 ? var : 0, st);
    // NDC of each chunk: the caller's statistics counter, read around the chunk
    static unsigned long long *own_stats[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    unsigned long long *cnt = a.stats;
    if (!cnt) {
        if (dev >= 64) return launch_dim_any(a, 0, st);
        if (!own_stats[dev] && cudaMalloc(&own_stats[dev], 2 * sizeof(unsigned long long)) != cudaSuccess)
            return launch_dim_any(a, 0, st);
        cnt = own_stats[dev];
    }
    double ms_of[kVariants] = {}, ndc_of[kVariants] = {};
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return launch_dim_any(a, 0, st);
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return launch_dim_any(a, 0, st);
    }
    cudaError_t err = cudaSuccess;
    unsigned long long before = 0, after = 0;
    for (int c = 0; c < kTuneChunks && err == cudaSuccess; ++c) {
        const int v = (c + c / kVariants) % kVariants;
        SearchArgs sl = subrange(a, a.nq * c / kTuneChunks, a.nq * (c + 1) / kTuneChunks);
        sl.stats = cnt;
        err = cudaMemcpyAsync(&before, cnt, sizeof(before), cudaMemcpyDeviceToHost, st);
        if (err == cudaSuccess) err = cudaMemsetAsync(a.work, 0, sizeof(int32_t), st);
        if (err == cudaSuccess) err = cudaEventRecord(e0, st);
        if (err == cudaSuccess) err = launch_dim_any(sl, v, st);
        if (err == cudaSuccess) err = cudaEventRecord(e1, st);
        if (err == cudaSuccess) err = cudaMemcpyAsync(&after, cnt, sizeof(after), cudaMemcpyDeviceToHost, st);
        if (err == cudaSuccess) err = cudaStreamSynchronize(st);
        float ms = 0.f;
        if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
        ms_of[v] += ms;
        ndc_of[v] += (double)(after - before);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err != cudaSuccess) return err;
    int best = 0;
    for (int v = 1; v < kVariants; ++v)
        if (ms_of[v] * ndc_of[best] < ms_of[best] * ndc_of[v]) best = v;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned[key] = best;
    return cudaSuccess;
}

bool search_dim_supported(int dim) {
    switch (dim) {
        case 8: case 16: case 32: case 64: case 96: case 128: case 256: case 768: return true;
        default: return false;
    }
}

}  // namespace rnsm
