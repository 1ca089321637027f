// Memory of the segmented BIT evaluation of f (host side): each segment of a
// tree needs its own Fenwick array (n int64: entries 1 .. n, 8-byte aligned)
// and its own DFS stack (stack_cap int4 entries, 16-byte aligned).  They are
// carved out of device memory regions the evaluation may reuse -- spare
// sub-wave slots, the stack buffer, walk arrays of rejected trees -- Fenwick
// arrays first, stacks in what the Fenwick arrays leave.  Plain C++ (no CUDA):
// the same header is compiled by the host tests.
#pragma once

#include <cstddef>
#include <cstdint>
#include <vector>

namespace kc_host {

struct SegRegion {
    uintptr_t p;   // device address
    size_t bytes;
};

// Carve `need` Fenwick arrays of bit_bytes and `need` stacks of stk_bytes from
// `regions`.  bits[i] is the 1-based base of Fenwick array i (its first byte
// minus 8, never dereferenced at index 0); stks[i] the first byte of stack i.
// Every slot lies inside one region and no two slots overlap.  Returns
// whether all fit (the vectors then hold exactly `need` entries each).
inline bool carve_segments(const std::vector<SegRegion> &regions, size_t need, size_t bit_bytes,
                           size_t stk_bytes, std::vector<uintptr_t> &bits,
                           std::vector<uintptr_t> &stks) {
    bits.clear();
    stks.clear();
    if (bit_bytes == 0 || stk_bytes == 0) return false;
    std::vector<uintptr_t> next(regions.size());
    for (size_t i = 0; i < regions.size(); ++i) {
        const uintptr_t e = regions[i].p + regions[i].bytes;
        uintptr_t a = (regions[i].p + 7) & ~(uintptr_t)7;
        while (bits.size() < need && a <= e && e - a >= bit_bytes) {
            bits.push_back(a - 8);
            a += bit_bytes;
        }
        next[i] = a;
    }
    if (bits.size() < need) return false;
    for (size_t i = 0; i < regions.size() && stks.size() < need; ++i) {
        const uintptr_t e = regions[i].p + regions[i].bytes;
        uintptr_t a = (next[i] + 15) & ~(uintptr_t)15;
        while (stks.size() < need && a <= e && e - a >= stk_bytes) {
            stks.push_back(a);
            a += stk_bytes;
        }
    }
    return stks.size() >= need;
}

// The largest k in [2, kmax] for which b k segments fit in `regions` (the
// slots are left in bits / stks), or 0 when not even two a tree fit.
inline int fit_segments(const std::vector<SegRegion> &regions, int64_t b, int kmax,
                        size_t bit_bytes, size_t stk_bytes, std::vector<uintptr_t> &bits,
                        std::vector<uintptr_t> &stks) {
    if (b <= 0) return 0;
    for (int k = kmax; k >= 2; --k)
        if (carve_segments(regions, (size_t)(b * k), bit_bytes, stk_bytes, bits, stks)) return k;
    bits.clear();
    stks.clear();
    return 0;
}

// The most segments per tree for a chunk of b trees under `ttf_segments`
// (kc_config): k >= 2 forces k, 1 never splits, 0 (automatic) splits only
// chunks evaluated after their wave's walk has ended (split while the walk
// runs, a chunk's warps slow the walker down), up to about 32 segment warps
// an SM (the residency of the segmented kernel) and at most 16 segments a
// tree.  0 or 1: no split.  The memory the chunk may use bounds it further.
inline int seg_limit(int ttf_segments, int64_t b, bool walk_over, int64_t num_sms) {
    if (ttf_segments >= 2) return ttf_segments;
    if (ttf_segments == 1 || !walk_over || b <= 0) return 0;
    const int64_t resident = num_sms > 0 ? 32 * num_sms : 32;
    const int64_t k = resident / b;
    return (int)(k < 16 ? k : 16);
}

}  // namespace kc_host
