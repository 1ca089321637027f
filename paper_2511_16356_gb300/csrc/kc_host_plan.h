// Wave planning for kc_sample (host side): how many trees a Wilson wave and a
// traversal sub-wave hold within a device-memory budget, and the workspace
// bytes a plan needs.
//
// Per tree of a Wilson wave: the walker words and the parent-first order
// (12 bytes a vertex).  Per tree of a traversal sub-wave: sizes, volumes and the
// DFN (16 bytes a vertex), the id-ordered sibling sums or preorder (4 more),
// and for the BIT evaluation of f the Fenwick array (8 more) -- its DFS stack is
// a separate allocation sized after the walk.  Low-eccentricity graphs (tau0
// scan) spend more time in the traversal than in the walk, so both get the same
// count; long-diameter graphs (BIT) spend most of it walking, which gets 70% of
// the budget by default (less when that would leave no room for one sub-wave
// tree).
//
// Plain C++ (no CUDA): the same header is compiled by the host tests.
#pragma once

#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdint>

namespace kc_host {

struct Plan {
    int64_t BW = 0;        // trees per Wilson wave
    int64_t BT = 0;        // trees per traversal sub-wave
    bool bit = false;
    int64_t stack_cap = 0; // BIT stack entries per tree
    bool canon = true;     // sub-wave buffers for the id-ordered DFN (aux array)
};

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Workspace bytes of a plan on an n-vertex graph (the layout carved from it).
inline size_t ws_bytes(int64_t n_vertices, const Plan &p) {
    const size_t n = (size_t)n_vertices;
    size_t b = 0;
    b += align256(sizeof(uint64_t) * n * p.BW);      // word
    b += align256(sizeof(int32_t) * n * p.BW);       // ord
    b += 3 * align256(sizeof(int64_t) * p.BW);       // steps, f, sids
    b += 2 * align256(sizeof(int32_t) * p.BW) + 256;  // hybrid hand-off: rs_q, rs_pos, done
    b += align256(sizeof(int32_t) * n * p.BT);       // size
    b += align256(sizeof(int64_t) * n * p.BT);       // vol
    b += align256(sizeof(int32_t) * n * p.BT);       // din
    if (p.bit || p.canon) b += align256(sizeof(int32_t) * n * p.BT);  // aux
    if (p.bit) b += align256(sizeof(int64_t) * (n + 1) * p.BT);  // bit
    return b;
}

// Wave sizes for ntrees trees within `budget` bytes (at least one tree each;
// max_in_flight > 0 caps the wave).  walker_share: the part of the budget the
// BIT variant gives to the Wilson wave (0.7; waves whose traversal streams
// through chunks of finished trees can give it more).
inline Plan plan_waves(int64_t n_vertices, int64_t ntrees, bool bit, bool canon, double budget,
                       int64_t max_in_flight, double walker_share = 0.7) {
    Plan p;
    p.bit = bit;
    p.canon = canon;
    const double n = (double)n_vertices;
    const double per_w = 12.0 * n + 64.0 + 8.0;
    const double per_t = (p.bit ? 28.0 : (canon ? 20.0 : 16.0)) * n + 64.0 +
                         (p.bit ? 16.0 * 4096.0 : 0.0);
    int64_t bw, bt;
    if (p.bit) {
        bw = (int64_t)std::floor(walker_share * budget / per_w);
        // leave room for at least one sub-wave tree
        bw = std::min<int64_t>(bw, (int64_t)std::floor((budget - per_t) / per_w));
        bw = std::max<int64_t>(1, std::min<int64_t>(bw, ntrees));
        if (max_in_flight > 0) bw = std::min(bw, max_in_flight);
        bw = std::min<int64_t>(bw, 1 << 20);
        bt = (int64_t)std::floor((budget - (double)bw * per_w) / per_t);
    } else {
        bw = (int64_t)std::floor(budget / (per_w + per_t));
        bw = std::max<int64_t>(1, std::min<int64_t>(bw, ntrees));
        if (max_in_flight > 0) bw = std::min(bw, max_in_flight);
        bw = std::min<int64_t>(bw, 1 << 20);
        bt = bw;
    }
    bt = std::max<int64_t>(1, std::min<int64_t>(bt, bw));
    bt = std::min<int64_t>(bt, 65535);
    p.BW = bw;
    p.BT = bt;
    p.stack_cap = p.bit ? 4096 : 0;
    return p;
}

// Trees a rejection wave draws so that it accepts `need` trees: need / rate
// plus three standard deviations of the accepted count, rate being the
// acceptance rate seen on the handle so far ((accepted + 1) / (drawn + 1),
// at least 1/64), or `hint` before any tree is seen.
inline int64_t reject_wave_size(int64_t need, int64_t drawn, int64_t accepted, double hint) {
    const double rate = drawn > 0 ? std::max(1.0 / 64.0, (double)(accepted + 1) /
                                                             (double)(drawn + 1))
                                  : hint;
    const double want = (double)need / rate;
    const double sd = std::sqrt(want * rate * (1.0 - rate)) / rate;
    return (int64_t)std::ceil(want + 3.0 * sd) + 8;
}

}  // namespace kc_host
