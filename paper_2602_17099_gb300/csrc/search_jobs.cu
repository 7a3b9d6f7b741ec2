// Multi-job launches of K1: one persistent launch searches the queries of
// many (source, target) pairs, each pair a job of the device job table.
#include "search_impl.cuh"

namespace rnsm {

cudaError_t launch_search_jobs(const SearchArgs &a, int var, cudaStream_t st) {
    return launch_dim<true>(a, var, st);
}

}  // namespace rnsm
