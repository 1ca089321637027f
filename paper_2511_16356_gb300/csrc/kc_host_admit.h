// Admission of waiting requests in the query server (host side).
//
// A waiting request may start when its graph has no request running, no
// earlier waiting request is on the same graph (requests on one graph run in
// submission order), and its workspace reservation fits the device budget
// beside the running requests' -- or nothing is running at all, so that a
// request larger than the budget still runs alone.  Later requests may pass
// one that does not fit yet.
//
// Plain C++ (no CUDA): the same header is compiled by the host tests.
#pragma once

#include <cstdint>
#include <vector>

namespace kc_host {

// Scans the waiting tickets [begin, end) in submission order and returns the
// first admissible one (end if none); *bytes receives its reservation.
// graph_of(ticket) -> graph index < n_graphs, busy(graph) -> bool,
// reserve(graph) -> bytes the request would reserve.
template <class It, class GraphOf, class Busy, class Reserve>
It first_admissible(It begin, It end, size_t n_graphs, GraphOf graph_of, Busy busy,
                    Reserve reserve, int64_t reserved, int64_t budget, int64_t *bytes) {
    std::vector<char> seen(n_graphs, 0);
    for (It it = begin; it != end; ++it) {
        const size_t gi = (size_t)graph_of(*it);
        if (seen[gi]) continue;  // an earlier request on this graph waits
        seen[gi] = 1;
        if (busy(gi)) continue;
        const int64_t b = reserve(gi);
        if (reserved + b > budget && reserved > 0) continue;
        *bytes = b;
        return it;
    }
    return end;
}

}  // namespace kc_host
