// rnsm_prune_noalloc: the occlusion prune without any device allocation.
//
// Some callers cannot let a library allocate device memory: services that
// hand all of HBM to their own pool allocator up front and leave no headroom
// for a library's cudaMalloc, and latency-critical paths that cannot afford
// the device-wide synchronisation cudaMalloc and cudaFree may imply.  This
// entry point runs the same prune kernels as rnsm_prune, but its scratch
// (work counters, error word, the list of owners handed from the small-pool
// kernel to the general one) lives in the file-scope array below, which every
// device that loads this library holds until the process exits.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "internal.h"
#include "rnsm.h"

namespace {

constexpr int64_t kMaxOwners = RNSM_PRUNE_NOALLOC_MAX_OWNERS;
constexpr size_t kHeadBytes = 256;  // err, two work counters, overflow count
constexpr size_t kScratchBytes = kHeadBytes + (size_t)kMaxOwners * sizeof(int32_t);

// Scratch shared by every call on a device.  In host code this name is only
// a stand-in for the device array: kernels get the address that
// cudaGetSymbolAddress returns for the current device.
static __device__ __align__(256) unsigned char g_prune_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
unsigned char *g_scratch_addr[kMaxDevices] = {};

// Once per device, with that device current: the device address of the array.
cudaError_t scratch_address(unsigned char **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_prune_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

rnsm_status fail(rnsm_status s, const char *msg) {
    rnsm::set_last_error(msg);
    return s;
}

rnsm_status cuda_fail(cudaError_t e, const char *what) {
    char buf[256];
    std::snprintf(buf, sizeof(buf), "%s: %s", what, cudaGetErrorString(e));
    rnsm::set_last_error(buf);
    return RNSM_ECUDA;
}

}  // namespace

extern "C" rnsm_status rnsm_prune_noalloc(const float *vecs, int64_t n, int32_t dim,
                                          const int32_t *owners, int64_t nv, const int32_t *pool,
                                          int32_t w_len, int32_t R, float alpha, int32_t metric,
                                          int32_t keep_all_if_fit, int32_t *out, void *stream) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (!vecs || n < 1 || n >= INT32_MAX) return fail(RNSM_EINVAL, "bad vectors or n");
    if (dim < 4 || (dim & 3) || dim > 1024) return fail(RNSM_EINVAL, "dim must be a multiple of 4 in [4, 1024]");
    if ((reinterpret_cast<uintptr_t>(vecs) & 15u) != 0) return fail(RNSM_EINVAL, "vectors must be 16-byte aligned");
    if (nv < 0 || (nv > 0 && (!owners || !out)) || w_len < 0 || w_len > 2048 ||
        (w_len > 0 && nv > 0 && !pool))
        return fail(RNSM_EINVAL, "bad owners, pool or output");
    if (nv > kMaxOwners)
        return fail(RNSM_EINVAL, "rnsm_prune_noalloc: nv exceeds the static scratch limit "
                                 "(RNSM_PRUNE_NOALLOC_MAX_OWNERS owners per call)");
    if (R < 1 || R > 64) return fail(RNSM_EINVAL, "R outside [1, 64]");
    if (!(std::isfinite(alpha) && alpha >= 0.f)) return fail(RNSM_EINVAL, "bad alpha");
    if (metric != 0 && metric != 1) return fail(RNSM_EINVAL, "unknown metric");
    if (nv == 0) return RNSM_OK;

    unsigned char *base = nullptr;
    cudaError_t e = scratch_address(&base);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress");
    int32_t *err = reinterpret_cast<int32_t *>(base);
    int32_t *work = reinterpret_cast<int32_t *>(base + 16);          // work, work2
    unsigned long long *ovf_count = reinterpret_cast<unsigned long long *>(base + 32);
    int32_t *ovf_list = reinterpret_cast<int32_t *>(base + kHeadBytes);

    // the array keeps the previous call's contents: zero the counters and the error word
    e = cudaMemsetAsync(base, 0, kHeadBytes, st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    if ((e = rnsm::launch_validate_vecs(vecs, n * dim, err, st)) != cudaSuccess ||
        (e = rnsm::launch_validate_ids(owners, nv, n, 0, err, st)) != cudaSuccess ||
        (w_len > 0 && (e = rnsm::launch_validate_ids(pool, nv * w_len, n, 1, err, st)) != cudaSuccess))
        return cuda_fail(e, "validation launch");
    int32_t herr = 0;
    if ((e = cudaMemcpyAsync(&herr, err, sizeof(herr), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return cuda_fail(e, "validation read-back");
    if (herr & 1) return fail(RNSM_EGRAPH, "an owner or pool id is outside its range");
    if (herr & 2) return fail(RNSM_EGRAPH, "vectors hold a non-finite value");

    rnsm::PruneArgs a;
    std::memset(&a, 0, sizeof(a));
    a.segs.base[0] = vecs;
    a.segs.off[1] = n;
    a.segs.m = 1;
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
    a.work = work;
    a.work2 = work + 1;
    a.ovf_list = ovf_list;
    a.ovf_count = ovf_count;
    a.err = err;
    if ((e = rnsm::launch_prune(a, st)) != cudaSuccess) return cuda_fail(e, "prune launch");
    if ((e = cudaMemcpyAsync(&herr, err, sizeof(herr), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return cuda_fail(e, "prune");
    if (herr & 16) return fail(RNSM_EGRAPH, "a prune pool exceeded 4096 candidates");
    if (herr) return fail(RNSM_ECUDA, "device error word set");
    return RNSM_OK;
}
