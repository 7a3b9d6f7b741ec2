// The multi-pair union variant of the merge (RNSM_FLAG_UNION): every plan edge
// is searched as in Algorithm 2, then each source vertex is pruned once over
// its list and the cross candidates of all its plan edges, and every target
// receives the reverse edges of all sources in one pass.  Two small kernels:
// the union pools of one source, and the kept cross edges of every source.
#include "internal.h"

namespace rnsm {

namespace {

// pool[v * (E c) + b c + j] = the j-th result of vertex v in edge b, as a global
// id (-1 stays -1)
__global__ void union_pool_kernel(UnionEdges e, int64_t ns, int32_t L, int32_t c, int32_t *pool) {
    const int64_t w = (int64_t)e.n * c;
    const int64_t total = ns * w;
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < total;
         x += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = x / w;
        const int32_t r = (int32_t)(x - v * w);
        const int32_t b = r / c, j = r - b * c;
        const int32_t u = e.res[b][v * L + j];
        pool[x] = u >= 0 ? u + e.t0[b] : -1;
    }
}

// For every vertex of a source segment (tmask[s] != 0) and every id u of its
// list whose segment is a target of s (bit seg(u) of tmask[s]): (u, v).
__global__ void emit_cross_kernel(const int32_t *lists, int32_t R, SegTable t, UnionMasks mk,
                                  int32_t *eu, int32_t *ev, unsigned long long *count) {
    const int64_t total = t.off[t.m] * R;
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < total;
         x += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = (int32_t)(x / R);
        const int32_t u = lists[x];
        bool e = false;
        if (u >= 0) {
            int sv = 0, su = 0;
            while (sv + 1 < t.m && t.off[sv + 1] <= v) ++sv;
            while (su + 1 < t.m && t.off[su + 1] <= u) ++su;
            e = (mk.tmask[sv] >> su) & 1ull;
        }
        if (e) {
            const unsigned long long slot = atomicAdd(count, 1ull);
            eu[slot] = u;
            ev[slot] = v;
        }
    }
}

unsigned grid_of(int64_t n) {
    int64_t g = (n + 255) / 256;
    if (g > 152 * 16) g = 152 * 16;
    return (unsigned)(g > 0 ? g : 1);
}

}  // namespace

cudaError_t launch_union_pool(const UnionEdges &e, int64_t ns, int32_t L, int32_t c, int32_t *pool,
                              cudaStream_t st) {
    if (ns <= 0 || e.n <= 0) return cudaSuccess;
    union_pool_kernel<<<grid_of(ns * e.n * c), 256, 0, st>>>(e, ns, L, c, pool);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_emit_cross(const int32_t *lists, int32_t R, const SegTable &t, const UnionMasks &mk,
                              int32_t *eu, int32_t *ev, unsigned long long *count, cudaStream_t st) {
    const int64_t total = t.off[t.m] * R;
    if (total <= 0) return cudaSuccess;
    emit_cross_kernel<<<grid_of(total), 256, 0, st>>>(lists, R, t, mk, eu, ev, count);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace rnsm
