// Host-side view of an undirected CSR graph with a batch of pending edge
// changes laid over it.  kc_update checks a whole batch against the evolving
// graph before applying anything (Sec. 4 takes one edge per update; a deleted
// edge must exist and must not be a bridge, an inserted one must not exist).
// The overlay answers those checks without copying or rebuilding the CSR:
// edge queries cost a hash lookup or a binary search in one row, and the
// bridge test searches from both endpoints of the deleted edge at once, so it
// stops as soon as the two searches meet (typically after a few hundred
// vertices) instead of traversing the whole graph.
//
// Plain C++ (no CUDA): the same header is compiled by the host tests.
#pragma once

#include <algorithm>
#include <cstdint>
#include <unordered_map>
#include <unordered_set>
#include <utility>
#include <vector>

namespace kc_host {

inline uint64_t edge_key(int32_t a, int32_t b) {
    if (a > b) std::swap(a, b);
    return ((uint64_t)(uint32_t)a << 32) | (uint64_t)(uint32_t)b;
}

class OverlayGraph {
  public:
    // row_off[n + 1] and col[2m]: the base graph, rows sorted ascending; the
    // arrays must outlive the overlay and are never written
    OverlayGraph(const int64_t *row_off, const int32_t *col, int64_t n)
        : ro_(row_off), col_(col), n_(n) {}

    bool has_edge(int32_t a, int32_t b) const {
        const uint64_t k = edge_key(a, b);
        if (added_.count(k)) return true;
        if (removed_.count(k)) return false;
        return base_has(a, b);
    }

    // precondition: a != b, the edge is absent
    void insert(int32_t a, int32_t b) {
        const uint64_t k = edge_key(a, b);
        if (removed_.erase(k)) return;  // a base edge deleted earlier in the batch
        added_.insert(k);
        extra_[a].push_back(b);
        extra_[b].push_back(a);
    }

    // precondition: the edge is present
    void erase(int32_t a, int32_t b) {
        const uint64_t k = edge_key(a, b);
        if (added_.erase(k)) {
            drop(extra_[a], b);
            drop(extra_[b], a);
            return;
        }
        removed_.insert(k);
    }

    // Whether a and b lie in one component of the current graph.  Two searches,
    // from a and from b, advance one vertex at a time on the side that has
    // discovered fewer vertices; they stop when one reaches a vertex the other
    // has seen (connected) or when one runs out of vertices (its whole
    // component is explored without meeting the other: not connected).
    bool connected(int32_t a, int32_t b) {
        if (a == b) return true;
        if (seen_.size() != (size_t)n_) seen_.assign((size_t)n_, 0);
        if (epoch_ >= 0x7FFFFFFFu - 2) {
            std::fill(seen_.begin(), seen_.end(), 0u);
            epoch_ = 0;
        }
        const uint32_t sa = ++epoch_, sb = ++epoch_;  // stamps of the two sides
        std::vector<int32_t> qa{a}, qb{b};
        size_t ha = 0, hb = 0;
        seen_[(size_t)a] = sa;
        seen_[(size_t)b] = sb;
        bool met = false;
        while (ha < qa.size() && hb < qb.size() && !met) {
            const bool side_a = qa.size() <= qb.size();
            std::vector<int32_t> &q = side_a ? qa : qb;
            size_t &h = side_a ? ha : hb;
            const uint32_t mine = side_a ? sa : sb, other = side_a ? sb : sa;
            const int32_t x = q[h++];
            for_each_neighbor(x, [&](int32_t y) {
                if (met) return;
                const uint32_t s = seen_[(size_t)y];
                if (s == other) {
                    met = true;
                } else if (s != mine) {
                    seen_[(size_t)y] = mine;
                    q.push_back(y);
                }
            });
        }
        return met;
    }

  private:
    bool base_has(int32_t a, int32_t b) const {
        const int32_t *first = col_ + ro_[a], *last = col_ + ro_[a + 1];
        return std::binary_search(first, last, b);
    }

    template <class F>
    void for_each_neighbor(int32_t x, F &&f) const {
        const bool any_removed = !removed_.empty();
        for (int64_t e = ro_[x]; e < ro_[x + 1]; ++e) {
            const int32_t y = col_[e];
            if (any_removed && removed_.count(edge_key(x, y))) continue;
            f(y);
        }
        auto it = extra_.find(x);
        if (it != extra_.end())
            for (int32_t y : it->second) f(y);
    }

    static void drop(std::vector<int32_t> &v, int32_t y) {
        auto it = std::find(v.begin(), v.end(), y);
        if (it != v.end()) {
            *it = v.back();
            v.pop_back();
        }
    }

    const int64_t *ro_;
    const int32_t *col_;
    int64_t n_;
    std::unordered_set<uint64_t> added_, removed_;
    std::unordered_map<int32_t, std::vector<int32_t>> extra_;
    std::vector<uint32_t> seen_;
    uint32_t epoch_ = 0;
};

}  // namespace kc_host
