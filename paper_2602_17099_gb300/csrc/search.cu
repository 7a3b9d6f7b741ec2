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

// Autotuner: the first launch with at least kTuneMin queries for a (dim,
// beam) shape runs every variant on the same slices of its queries: one
// untimed warm-up slice, then kTuneReps timed slices, each run by every
// variant in turn (order alternating between slices; CUDA events on the
// launching stream).  The variant with the smallest total time is kept for
// later launches.  Every variant computes the same results, so running a
// slice again only costs time, and the comparison is on identical work.
constexpr int64_t kTuneWarm = 2000;
constexpr int64_t kTuneSlice = 8000;
constexpr int kTuneReps = 3;
constexpr int64_t kTuneMin = kTuneWarm + kTuneReps * kTuneSlice + 10000;
std::mutex g_tune_mu;
std::map<std::pair<int, int>, int> g_tuned;

int efmax_of(int ef) { return ef <= 32 ? 32 : ef <= 64 ? 64 : ef <= 128 ? 128 : 256; }

}  // namespace

int search_variant_for(int dim, int ef) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tuned.find({dim, efmax_of(ef)});
    return it == g_tuned.end() ? -1 : it->second;
}

bool search_would_tune(int dim, int ef, int64_t nq) {
    const char *force = getenv("RNSM_SEARCH_VARIANT");
    if (force && force[0] >= '0' && force[0] < '0' + kVariants) return false;
    if (nq < kTuneMin) return false;
    return search_variant_for(dim, ef) < 0;
}

cudaError_t launch_search(const SearchArgs &a, cudaStream_t st) {
    if (a.nq <= 0) return cudaSuccess;
    if (!search_dim_supported(a.dim)) return cudaErrorInvalidValue;
    const char *force = getenv("RNSM_SEARCH_VARIANT");
    if (force && force[0] >= '0' && force[0] < '0' + kVariants) return launch_dim_any(a, force[0] - '0', st);
    const std::pair<int, int> key{a.dim, efmax_of(a.ef)};
    int var = -1;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tuned.find(key);
        if (it != g_tuned.end()) var = it->second;
    }
    if (var >= 0 || a.nq < kTuneMin) return launch_dim_any(a, var >= 0 ? var : 0, st);
    // every variant runs each slice; the slices' results are final
    float total_ms[kVariants];
    for (int v = 0; v < kVariants; ++v) total_ms[v] = 0.f;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return launch_dim_any(a, 0, st);
    cudaError_t err = cudaSuccess;
    int64_t pos = 0;
    auto run_slice = [&](int v, int64_t len, bool timed) {
        const SearchArgs sl = subrange(a, pos, pos + len);
        err = cudaMemsetAsync(a.work, 0, sizeof(int32_t), st);  // each run starts its own count
        if (err != cudaSuccess) return;
        if (timed) cudaEventRecord(e0, st);
        err = launch_dim_any(sl, v, st);
        if (err != cudaSuccess || !timed) return;
        cudaEventRecord(e1, st);
        err = cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        total_ms[v] += ms;
    };
    for (int v = 0; v < kVariants && err == cudaSuccess; ++v) run_slice(v, kTuneWarm, false);
    pos += kTuneWarm;
    for (int rep = 0; rep < kTuneReps && err == cudaSuccess; ++rep) {
        for (int k = 0; k < kVariants && err == cudaSuccess; ++k)
            run_slice(rep % 2 == 0 ? k : kVariants - 1 - k, kTuneSlice, true);
        pos += kTuneSlice;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err != cudaSuccess) return err;
    int best = 0;
    for (int v = 1; v < kVariants; ++v)
        if (total_ms[v] < total_ms[best]) best = v;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tuned[key] = best;
    }
    err = cudaMemsetAsync(a.work, 0, sizeof(int32_t), st);
    if (err != cudaSuccess) return err;
    return launch_dim_any(subrange(a, pos, a.nq), best, st);
}

bool search_dim_supported(int dim) {
    switch (dim) {
        case 8: case 16: case 32: case 64: case 96: case 128: case 256: case 768: return true;
        default: return false;
    }
}

}  // namespace rnsm
