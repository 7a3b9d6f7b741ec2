// Host planners of the merge: lazy-greedy pivot selection (Algorithm 2,
// Phase 2) and Merge Order Selection (Algorithm 3) with the execution order
// of its edges (Section 5).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <queue>
#include <vector>

#include "host.h"

namespace rnsm {

namespace {

struct HeapItem {
    int64_t gain;
    int32_t x;
};

// Max-heap on gain; equal gains pop the lower id first.
struct HeapLess {
    bool operator()(const HeapItem &a, const HeapItem &b) const {
        if (a.gain != b.gain) return a.gain < b.gain;
        return a.x > b.x;
    }
};

}  // namespace

int64_t select_pivots_host(int64_t n, const int64_t *offs, const int32_t *ids, int32_t *pivot_of,
                           std::vector<int32_t> &pivots) {
    std::vector<uint8_t> covered((size_t)n, 0);
    std::vector<HeapItem> init;
    init.reserve((size_t)n);
    for (int64_t x = 0; x < n; ++x) {
        init.push_back({offs[x + 1] - offs[x], (int32_t)x});
        pivot_of[x] = -1;
    }
    std::priority_queue<HeapItem, std::vector<HeapItem>, HeapLess> heap(HeapLess(),
                                                                         std::move(init));
    pivots.clear();
    while (!heap.empty()) {
        const HeapItem top = heap.top();
        heap.pop();
        const int32_t x = top.x;
        if (covered[x]) continue;
        int64_t gain = 0;
        for (int64_t e = offs[x]; e < offs[x + 1]; ++e) gain += covered[ids[e]] ? 0 : 1;
        if (gain < top.gain) {  // stale upper bound: reinsert with the current gain
            heap.push({gain, x});
            continue;
        }
        for (int64_t e = offs[x]; e < offs[x + 1]; ++e) {
            const int32_t y = ids[e];
            if (!covered[y]) {
                covered[y] = 1;
                pivot_of[y] = x;  // follower of x
            }
        }
        covered[x] = 1;
        pivot_of[x] = -1;
        pivots.push_back(x);
    }
    return (int64_t)pivots.size();
}

namespace {

constexpr int32_t kFar = 1 << 29;

void all_pairs_hops(int32_t m, const std::vector<uint8_t> &adj, std::vector<int32_t> &hop) {
    std::vector<int32_t> queue((size_t)m);
    for (int32_t s = 0; s < m; ++s) {
        int32_t *h = &hop[(size_t)s * m];
        std::fill(h, h + m, kFar);
        h[s] = 0;
        int32_t head = 0, tail = 0;
        queue[tail++] = s;
        while (head < tail) {
            const int32_t a = queue[head++];
            for (int32_t b = 0; b < m; ++b)
                if (adj[(size_t)a * m + b] && h[b] == kFar) {
                    h[b] = h[a] + 1;
                    queue[tail++] = b;
                }
        }
    }
}

}  // namespace

bool mos_greedy(int32_t m, const std::vector<double> &C, int32_t Rm, int32_t Delta,
                std::vector<std::pair<int32_t, int32_t>> &edges) {
    edges.clear();
    // Vertices by ascending mean cost to their Rm cheapest others (ties: index).
    std::vector<double> mean((size_t)m, 0.0);
    for (int32_t i = 0; i < m; ++i) {
        std::vector<double> row;
        for (int32_t j = 0; j < m; ++j)
            if (j != i) row.push_back(C[(size_t)i * m + j]);
        std::sort(row.begin(), row.end());
        const size_t take = std::min<size_t>(row.size(), (size_t)Rm);
        double s = 0.0;
        for (size_t t = 0; t < take; ++t) s += row[t];
        mean[i] = take ? s / (double)take : 0.0;
    }
    std::vector<int32_t> order((size_t)m);
    for (int32_t i = 0; i < m; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(),
                     [&](int32_t a, int32_t b) { return mean[a] < mean[b]; });

    std::vector<uint8_t> adj((size_t)m * m, 0);
    std::vector<int32_t> deg((size_t)m, 0), hop((size_t)m * m);
    all_pairs_hops(m, adj, hop);
    auto cost = [&](int32_t a, int32_t b) { return C[(size_t)a * m + b]; };
    // Cheapest neighbour y of `hub` below the bound, not `other` nor adjacent to it.
    auto relay = [&](int32_t hub, int32_t other) {
        int32_t best = -1;
        for (int32_t y = 0; y < m; ++y) {
            if (!adj[(size_t)hub * m + y] || y == other || adj[(size_t)other * m + y] ||
                deg[y] >= Rm)
                continue;
            if (best < 0 || cost(y, other) < cost(best, other)) best = y;
        }
        return best;
    };
    for (int32_t v : order) {
        for (;;) {
            int32_t x = -1;
            for (int32_t j = 0; j < m; ++j)
                if (j != v && hop[(size_t)v * m + j] > Delta && (x < 0 || cost(v, j) < cost(v, x)))
                    x = j;
            if (x < 0) break;
            int32_t a = v, b = x;
            const bool sv = deg[v] >= Rm, sx = deg[x] >= Rm;
            if (!sv && sx && Delta >= 2) {
                const int32_t y = relay(x, v);
                if (y >= 0) b = y;
            } else if (sv && !sx && Delta >= 2) {
                const int32_t y = relay(v, x);
                if (y >= 0) a = y;
            }
            // both saturated (or no relay): the direct edge keeps connectivity
            adj[(size_t)a * m + b] = adj[(size_t)b * m + a] = 1;
            ++deg[a];
            ++deg[b];
            edges.emplace_back(a, b);
            all_pairs_hops(m, adj, hop);
        }
    }
    return true;
}

int32_t mos_plan_host(int32_t m, const int64_t *sizes, const float *centroids, int32_t D,
                      int32_t Rm, int32_t Delta, std::vector<PlanEdge> &plan) {
    plan.clear();
    if (Rm <= 0) {
        int32_t r = 0;
        while ((int64_t)r * r < (int64_t)(m - 1)) ++r;
        Rm = r + 1;
    }
    if (Delta <= 0) Delta = 2;
    std::vector<double> C((size_t)m * m, 0.0);
    for (int32_t i = 0; i < m; ++i)
        for (int32_t j = 0; j < m; ++j) {
            if (i == j) continue;
            if (!centroids) {
                C[(size_t)i * m + j] = 1.0;
                continue;
            }
            double s = 0.0;
            for (int32_t t = 0; t < D; ++t) {
                const double z = (double)centroids[(size_t)i * D + t] - (double)centroids[(size_t)j * D + t];
                s += z * z;
            }
            C[(size_t)i * m + j] = std::sqrt(s);
        }
    std::vector<std::pair<int32_t, int32_t>> edges;
    mos_greedy(m, C, Rm, Delta, edges);
    for (auto &e : edges) {
        const int32_t lo = std::min(e.first, e.second), hi = std::max(e.first, e.second);
        plan.push_back({lo, hi, C[(size_t)lo * m + hi]});
    }
    // closer pairs first; ties by (min index, max index)
    std::stable_sort(plan.begin(), plan.end(), [](const PlanEdge &a, const PlanEdge &b) {
        if (a.cost != b.cost) return a.cost < b.cost;
        if (a.src != b.src) return a.src < b.src;
        return a.dst < b.dst;
    });
    // orient: smaller segment merges into the larger; equal sizes: larger index is the source
    for (auto &e : plan) {
        const int32_t lo = e.src, hi = e.dst;
        if (sizes[lo] < sizes[hi]) {
            e.src = lo;
            e.dst = hi;
        } else {
            e.src = hi;
            e.dst = lo;
        }
    }
    return (int32_t)plan.size();
}

}  // namespace rnsm
