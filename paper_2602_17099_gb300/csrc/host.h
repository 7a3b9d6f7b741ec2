// Host planners (pivot selection, MOS).
#pragma once

#include <cstdint>
#include <utility>
#include <vector>

namespace rnsm {

struct PlanEdge {
    int32_t src;
    int32_t dst;
    double cost;
};

// Lazy greedy of Algorithm 2 (Phase 2).  pivot_of[y] = pivot of follower y,
// -1 for pivots; pivots in selection order.  Returns the pivot count.
int64_t select_pivots_host(int64_t n, const int64_t *offs, const int32_t *ids, int32_t *pivot_of,
                           std::vector<int32_t> &pivots);

// Algorithm 3 on a symmetric cost matrix; edges in insertion order.
bool mos_greedy(int32_t m, const std::vector<double> &C, int32_t Rm, int32_t Delta,
                std::vector<std::pair<int32_t, int32_t>> &edges);

// Cost matrix, Algorithm 3, execution order and orientation.
int32_t mos_plan_host(int32_t m, const int64_t *sizes, const float *centroids, int32_t D,
                      int32_t Rm, int32_t Delta, std::vector<PlanEdge> &plan);

}  // namespace rnsm
