// Static work schedules built on the host (plain C++, no CUDA types, so the
// host tests compile it on its own).
#pragma once
#include <stdint.h>
#include <algorithm>
#include <functional>
#include <numeric>
#include <queue>
#include <utility>
#include <vector>

namespace bddc {

// Groups `items` into `nbins` bins of near-equal total cost: the items go, the
// most expensive first (equal costs in their given order), onto the bin with the
// least cost so far (ties to the lower bin index).  This greedy rule ends within
// (4/3 - 1/(3 nbins)) of the best possible largest bin (Graham's bound for
// longest-processing-time-first scheduling).  On return `out` holds the items
// bin by bin, each bin keeping the items' given relative order, and bin b is
// out[binptr[b] .. binptr[b + 1]).  `cost(item)` returns a non-negative int64_t.
template <class Item, class Cost>
void bin_by_cost(const std::vector<Item> &items, Cost cost, int nbins, std::vector<Item> &out,
                 std::vector<int> &binptr) {
    const int m = std::max(nbins, 1);
    std::vector<int64_t> c(items.size());
    for (size_t k = 0; k < items.size(); ++k) c[k] = (int64_t)cost(items[k]);
    std::vector<int> order(items.size());
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return c[a] > c[b]; });
    using Load = std::pair<int64_t, int>;
    std::priority_queue<Load, std::vector<Load>, std::greater<Load>> q;
    for (int b = 0; b < m; ++b) q.push({0, b});
    std::vector<int> bin_of(items.size());
    for (int k : order) {
        Load l = q.top();
        q.pop();
        bin_of[k] = l.second;
        q.push({l.first + c[k], l.second});
    }
    binptr.assign(m + 1, 0);
    for (size_t k = 0; k < items.size(); ++k) ++binptr[bin_of[k] + 1];
    for (int b = 0; b < m; ++b) binptr[b + 1] += binptr[b];
    std::vector<int> fill(binptr.begin(), binptr.end() - 1);
    out.resize(items.size());
    for (size_t k = 0; k < items.size(); ++k) out[fill[bin_of[k]]++] = items[k];
}

}  // namespace bddc
