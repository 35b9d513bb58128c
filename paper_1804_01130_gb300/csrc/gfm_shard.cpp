// Sharding a batch of independent tanks over several GPUs (one process per
// GPU).  The tanks of a batch share nothing -- each is its own pressure
// equation (Sec. 3.1) with its own pin -- so they split across ranks with no
// exchange on the data path: every rank builds a batched handle of its own
// tanks, and only the per-tank solve records are gathered at the end.
//
// The split balances cells, the work of one CG iteration: longest
// processing time first (tanks in descending cell count, ties by tank
// index), each onto the rank with the least cells so far (ties to the lower
// rank).  The result is a pure function of the cell counts and the rank
// count, so every rank computes the same table without communicating.  List
// scheduling bounds the busiest rank by total/ranks + (1 - 1/ranks) * largest.
#include <algorithm>
#include <cstdint>
#include <numeric>
#include <vector>

#include "gfm.h"

extern "C" gfm_status gfm_partition_tanks(const int64_t *cells, int32_t n_tanks, int32_t n_ranks,
                                          int32_t *rank_of_tank, int64_t *rank_cells)
{
    if (!cells || !rank_of_tank || n_tanks < 1 || n_ranks < 1) return GFM_ERR_ARG;
    for (int32_t t = 0; t < n_tanks; ++t)
        if (cells[t] < 1) return GFM_ERR_ARG;
    std::vector<int32_t> order((size_t)n_tanks);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return cells[a] > cells[b]; });
    std::vector<int64_t> load((size_t)n_ranks, 0);
    for (int32_t t : order) {
        int32_t best = 0;
        for (int32_t r = 1; r < n_ranks; ++r)
            if (load[(size_t)r] < load[(size_t)best]) best = r;
        rank_of_tank[t] = best;
        load[(size_t)best] += cells[t];
    }
    if (rank_cells)
        for (int32_t r = 0; r < n_ranks; ++r) rank_cells[r] = load[(size_t)r];
    return GFM_OK;
}
