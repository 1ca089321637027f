// Wilson's loop-erased-walk sampler (Sec. 2.2; Algorithm 1, "wilson(G, r)").
//
// One lane owns one tree.  The lane runs Wilson's algorithm as a flat state
// machine (SEEK a start vertex outside the tree, WALK, count the loop-erased
// path, commit it) so that every loop iteration issues at most one dependent
// gather and the warp re-converges every iteration.  The departure of u on its
// k-th visit follows neighbour bounded(seed, u, k, sample, WALK, deg u): loop
// erasure is implicit (next[u] is overwritten on the next departure) and the
// resulting tree and step count do not depend on the start order.
//
// Per step the lane touches one 32-byte vertex record (degree, offset and the
// first neighbours) and the 8-byte walker word of the next vertex; both loads
// are issued together.  Committing a path of length L writes the words with
// the in-tree flag and depth and the path, parent first, into `ord`.
#include "kc_common.cuh"

namespace kc {

namespace {

enum : int { kSeek = 0, kWalk = 1, kCount = 2, kCommit = 3, kDone = 4 };

__global__ void k_wave_init(int64_t n, int64_t B, int32_t root, uint64_t *word, int32_t *ord) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= B) return;
    word[t * n + root] = w_make(-1, 0, true);
    ord[t * n] = root;
}

__global__ void __launch_bounds__(128) k_wilson(GraphView g, WaveView w, uint64_t seed,
                                                const int64_t *__restrict__ sids,
                                                int64_t step_cap) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= w.B) return;
    const int64_t n = g.n;
    uint64_t *__restrict__ word = w.word + t * n;
    int32_t *__restrict__ ord = w.ord + t * n;
    const VRec *__restrict__ rec = g.rec;
    const uint32_t sample = (uint32_t)sids[t];

    int64_t steps = 0;
    int32_t pos = w.pos0;  // ord[0 .. pos0) already placed (the root, or an edge)
    int32_t s = 0;         // current start vertex
    int32_t u = 0;         // walker position (WALK) / path cursor (COUNT, COMMIT)
    uint64_t wu = 0;       // word of u (WALK)
    VRec ru;               // record of u (WALK)
    int32_t len = 0, i = 0, dh = 0, maxd = 0;
    int phase = kSeek;

    while (phase != kDone) {
        if (phase == kSeek) {
            if (s >= n) { phase = kDone; break; }
            const uint64_t ws = word[s];
            if (w_in_tree(ws)) { ++s; continue; }
            u = s;
            wu = ws;
            ru = rec[s];
            phase = kWalk;
        } else if (phase == kWalk) {
            const uint32_t k = bounded_draw(seed, (uint32_t)u, w_count(wu), sample, kTagWalk,
                                            (uint32_t)ru.deg);
            int32_t v;
            if (k < (uint32_t)kInline) {
                // register select instead of a dynamic index into the record
                v = ru.nbr[0];
#pragma unroll
                for (int q = 1; q < kInline; ++q) v = (k == (uint32_t)q) ? ru.nbr[q] : v;
            } else {
                const uint64_t off = (uint64_t)ru.off_lo | ((uint64_t)ru.off_hi << 32);
                v = g.col[off + k];
            }
            word[u] = w_make(v, w_count(wu) + 1, false);
            if (++steps > step_cap) {
                atomicOr(w.err, kErrStepLimit);
                phase = kDone;
                break;
            }
            const uint64_t wv = word[v];
            const VRec rv = load_rec(rec + v);
            if (w_in_tree(wv)) {
                u = s;
                len = 0;
                phase = kCount;
            } else {
                u = v;
                wu = wv;
                ru = rv;
            }
        } else if (phase == kCount) {
            // length of the loop-erased path from s and the depth of its tree end
            const uint64_t wx = word[u];
            if (w_in_tree(wx)) {
                dh = (int32_t)w_count(wx);
                u = s;
                i = 0;
                phase = kCommit;
            } else {
                ++len;
                u = w_next(wx);
                if (len > n || u < 0 || u >= n) {  // a path longer than n means corrupt state
                    atomicOr(w.err, kErrBadTree);
                    phase = kDone;
                    break;
                }
            }
        } else {  // kCommit
            const uint64_t wx = word[u];
            const int32_t nx = w_next(wx);
            const int32_t d = dh + len - i;
            word[u] = w_make(nx, (uint32_t)d, true);
            ord[pos + len - 1 - i] = u;
            if (d > maxd) maxd = d;
            ++i;
            u = nx;
            if (i == len) {
                pos += len;
                ++s;
                phase = kSeek;
            }
        }
    }
    w.steps[t] = steps;
    atomicMax(w.maxdepth, maxd);
}

// ---------------------------------------------------------------------------
// Warp-cooperative variant: the 32 lanes of a warp are 32 concurrent walkers of
// ONE tree.  Wilson's algorithm equals cycle popping on the stacks of arrows
// (vertex u's k-th arrow is fixed by (u, k)), and popping cycles in any order
// yields the same tree and the same number of revealed arrows.  The walkers only
// ever pop genuine cycles of the current arrow graph:
//   - a walker owns the vertices of its live path (ownership is stored in the
//     vertex word), departs only from its own frontier and claims free
//     vertices (a free vertex has no live arrow);
//   - closing a loop on its own path frees the loop (all but the entry vertex,
//     which is re-departed);
//   - a walker whose arrow points into another walker's path waits; waits that
//     close a cycle among walkers form a cycle of arrows, which is popped: each
//     walker frees its segment after the vertex its predecessor waits on and
//     re-departs from that vertex;
//   - a path whose arrows reach the tree is committed (in-tree flag, depth,
//     parent-first order).
// Everything is warp-synchronous: one memory action per lane per iteration,
// claims resolved with __match_any_sync (lowest lane wins), wait cycles found
// by pointer chasing over shuffles.  No lane ever spins on another warp.
//
// Word of a vertex outside the tree: bits 0..31 next, 32..56 departures,
// 57..61 owner lane, 62 owned; in-tree words are as in the lane variant.
// ---------------------------------------------------------------------------
constexpr uint64_t kOwned = 1ull << 62;
constexpr uint32_t kCountMask = (1u << 25) - 1u;

__device__ __forceinline__ bool o_owned(uint64_t w) { return (w & kOwned) != 0; }
__device__ __forceinline__ int o_owner(uint64_t w) { return (int)((w >> 57) & 31u); }
__device__ __forceinline__ uint32_t o_count(uint64_t w) {
    return (uint32_t)(w >> 32) & kCountMask;
}
__device__ __forceinline__ uint64_t o_free(int32_t next, uint32_t count) {
    return (uint64_t)(uint32_t)next | ((uint64_t)(count & kCountMask) << 32);
}
__device__ __forceinline__ uint64_t o_own(int32_t next, uint32_t count, int lane) {
    return o_free(next, count) | ((uint64_t)lane << 57) | kOwned;
}
__device__ __forceinline__ int32_t rec_neighbor(const VRec &r, const int32_t *col, uint32_t k) {
    if (k < (uint32_t)kInline) {
        int32_t v = r.nbr[0];
#pragma unroll
        for (int q = 1; q < kInline; ++q) v = (k == (uint32_t)q) ? r.nbr[q] : v;
        return v;
    }
    const uint64_t off = (uint64_t)r.off_lo | ((uint64_t)r.off_hi << 32);
    return col[off + k];
}
__device__ __forceinline__ uint64_t ld_word(const uint64_t *p) {
    return (uint64_t)__ldcg((const unsigned long long *)p);
}
__device__ __forceinline__ void st_word(uint64_t *p, uint64_t v) {
    __stcg((unsigned long long *)p, (unsigned long long)v);
}

enum : int {
    pIdle = 0,     // needs a start vertex
    pWalk = 1,     // owns frontier c and departs from it
    pWait = 2,     // arrow (or empty path) points at x, owned by another lane
    pArrive = 3,   // reload frontier c (word and record) before walking
    pPopSet = 4,   // read the re-departure vertex before freeing a popped segment
    pPop = 5,      // free the vertices pcur .. pend of a popped cycle
    pCount = 6,    // length of the committed path
    pCommit = 7,   // write in-tree words, depths and the parent-first order
    pDone = 8
};

__global__ void __launch_bounds__(128) k_wilson_warp(GraphView g, WaveView w, uint64_t seed,
                                                     const int64_t *__restrict__ sids,
                                                     const int32_t *__restrict__ sorder,
                                                     int64_t step_cap, int64_t iter_cap) {
    const unsigned kFull = 0xFFFFFFFFu;
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (t >= w.B) return;  // whole warp
    const int64_t n = g.n;
    uint64_t *word = w.word + t * n;
    int32_t *ord = w.ord + t * n;
    const VRec *__restrict__ rec = g.rec;
    const uint32_t sample = (uint32_t)sids[t];

    int ph = pIdle;
    bool has_path = false;
    int32_t s = -1, c = -1, x = -1, u = -1, pcur = -1, pend = -1, prew = -1;
    uint32_t cc = 0, prew_cc = 0;
    VRec rc;
    rc.deg = 1;
    int32_t len = 0, i = 0, dh = 0, mypos = 0, maxd = 0;
    int64_t steps = 0;
    int64_t next_start = 0;  // warp-uniform
    int64_t pos = w.pos0;    // warp-uniform, ord[0 .. pos0) already placed
    bool bad = false;

    for (int64_t it = 0;; ++it) {
        // ---- hand out start vertices to idle lanes
        const unsigned idle = __ballot_sync(kFull, ph == pIdle);
        if (idle) {
            if (ph == pIdle) {
                const int64_t q = next_start + __popc(idle & lt);
                if (q < n) s = sorder[q]; else ph = pDone;
                has_path = false;
            }
            next_start += __popc(idle);
        }
        if (__all_sync(kFull, ph == pDone)) break;
        if (it > iter_cap || __any_sync(kFull, bad)) {
            if (lane == 0) atomicOr(w.err, bad ? kErrBadTree : kErrIterLimit);
            break;
        }
        // ---- act: departures and the address each lane reads this iteration
        int32_t ld = -1;
        if (ph == pWalk) {
            const uint32_t k = bounded_draw(seed, (uint32_t)c, cc, sample, kTagWalk,
                                            (uint32_t)rc.deg);
            const int32_t v = rec_neighbor(rc, g.col, k);
            st_word(word + c, o_own(v, cc + 1, lane));
            cc += 1;
            ++steps;
            if (cc >= kCountMask || steps > step_cap) {
                atomicOr(w.err, kErrStepLimit);
                bad = true;
            }
            x = v;
            ld = v;
        } else if (ph == pIdle) {
            ld = s;
        } else if (ph == pWait) {
            ld = x;
        } else if (ph == pArrive) {
            ld = c;
        } else if (ph == pPopSet) {
            ld = prew;
        } else if (ph == pPop) {
            ld = pcur;
        } else if (ph == pCount || ph == pCommit) {
            ld = u;
        }
        __syncwarp();
        uint64_t wl = 0;
        VRec rl;
        rl.deg = 1;
        if (ld >= 0) wl = ld_word(word + ld);
        const bool may_walk = (ph == pIdle || ph == pWalk || ph == pWait);
        if ((may_walk || ph == pArrive) && ld >= 0) rl = rec[ld];
        // ---- resolve
        const bool inT = w_in_tree(wl);
        const bool own = !inT && o_owned(wl);
        const int ownr = o_owner(wl);
        const bool was_wait = (ph == pWait);
        const bool want = may_walk && ld >= 0 && !inT && !own;
        const unsigned grp = __match_any_sync(kFull, want ? ld : -1 - lane);
        bool fin = false;
        if (want) {
            if (lane == __ffs(grp) - 1) {  // the claim goes to the lowest lane
                st_word(word + ld, o_own(w_next(wl), o_count(wl), lane));
                if (!has_path) s = ld;
                has_path = true;
                c = ld;
                cc = o_count(wl);
                rc = rl;
                ph = pWalk;
            } else {
                if (ph == pIdle) has_path = false;
                x = ld;
                ph = pWait;
            }
        } else if (may_walk && ld >= 0) {
            if (inT) {
                if (!has_path) {
                    ph = pIdle;
                } else {
                    ph = pCount;
                    u = s;
                    len = 0;
                }
            } else if (ownr == lane) {
                // loop closed on the own path: free next(ld) .. c, re-depart from ld
                prew = ld;
                prew_cc = o_count(wl);
                pcur = w_next(wl);
                pend = c;
                ph = pPop;
            } else {
                if (ph == pIdle) has_path = false;
                x = ld;
                ph = pWait;
            }
        } else if (ph == pArrive) {
            cc = o_count(wl);
            rc = rl;
            ph = pWalk;
        } else if (ph == pPopSet) {
            prew_cc = o_count(wl);
            if (prew == c) {
                cc = prew_cc;  // c's record is still in rc
                ph = pWalk;
            } else {
                pcur = w_next(wl);
                pend = c;
                ph = pPop;
            }
        } else if (ph == pPop) {
            const int32_t nx = w_next(wl);
            st_word(word + pcur, o_free(nx, o_count(wl)));
            if (pcur == pend) {
                c = prew;
                ph = pArrive;
            } else {
                pcur = nx;
                if (pcur < 0 || pcur >= n) bad = true;
            }
        } else if (ph == pCount) {
            if (inT) {
                dh = (int32_t)w_count(wl);
                fin = true;
            } else {
                ++len;
                u = w_next(wl);
                if (len > n || u < 0 || u >= n) bad = true;
            }
        } else if (ph == pCommit) {
            const int32_t nx = w_next(wl);
            const int32_t d = dh + len - i;
            st_word(word + u, w_make(nx, (uint32_t)d, true));
            const int64_t slot = (int64_t)mypos + len - 1 - i;
            if (slot > 0 && slot < n) ord[slot] = u; else bad = true;
            if (d > maxd) maxd = d;
            ++i;
            u = nx;
            if (i == len) ph = pIdle;
        }
        // ---- reserve slots of the parent-first order for paths that reached the tree
        {
            int32_t v = fin ? len : 0;
            int32_t incl = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int32_t y = __shfl_up_sync(kFull, incl, o);
                if (lane >= o) incl += y;
            }
            const int32_t total = __shfl_sync(kFull, incl, 31);
            if (fin) {
                mypos = (int32_t)pos + incl - v;
                ph = pCommit;
                u = s;
                i = 0;
            }
            pos += total;
        }
        // ---- wait cycles: each lane that stays waiting points at the owner of its target
        // (a cycle of waits persists until it is popped, so looking every 4th
        // iteration only delays the pop a little and saves the shuffle chains)
        const int succ = (was_wait && ph == pWait && has_path && own && ownr != lane) ? ownr : -1;
        const unsigned wm = __ballot_sync(kFull, succ >= 0);
        if ((it & 3) == 0 && __popc(wm) >= 2) {
            int y = lane;
            bool on = false;
#pragma unroll 4
            for (int k = 0; k < 32; ++k) {
                const int sy = __shfl_sync(kFull, succ, y < 0 ? lane : y);
                y = (y < 0) ? -1 : sy;
                if (y == lane) on = true;
            }
            on = on && succ >= 0;
            const unsigned onm = __ballot_sync(kFull, on);
            if (onm) {
                int pred = -1;
                for (int j = 0; j < 32; ++j) {
                    const int sj = __shfl_sync(kFull, succ, j);
                    if (((onm >> j) & 1u) && sj == lane) pred = j;
                }
                const int32_t xp = __shfl_sync(kFull, x, pred < 0 ? lane : pred);
                if (on) {
                    // the vertex my predecessor waits on is on my path: pop the
                    // cycle segment after it and re-depart from it
                    prew = xp;
                    ph = pPopSet;
                }
            }
        }
    }
    long long tot = (long long)steps;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) tot += __shfl_down_sync(kFull, tot, o);
    int md = maxd;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) md = max(md, __shfl_down_sync(kFull, md, o));
    if (lane == 0) {
        w.steps[t] = tot;
        atomicMax(w.maxdepth, md);
    }
}

}  // namespace

cudaError_t launch_wilson_warp(const GraphView &g, WaveView w, uint64_t seed, const int64_t *sids,
                               const int32_t *sorder, int64_t step_cap, cudaStream_t s) {
    // a correct run needs at most about 3 iterations per departure (walk,
    // count, commit / pop), however the walkers serialise
    const int64_t iter_cap = 4 * step_cap + 64 * g.n + 4096;
    k_wilson_warp<<<(unsigned)((w.B * 32 + 127) / 128), 128, 0, s>>>(g, w, seed, sids, sorder,
                                                                      step_cap, iter_cap);
    return cudaGetLastError();
}

cudaError_t launch_wave_init(const GraphView &g, WaveView w, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(w.word, 0, sizeof(uint64_t) * (size_t)(w.B * g.n), s);
    if (e != cudaSuccess) return e;
    k_wave_init<<<(unsigned)((w.B + 127) / 128), 128, 0, s>>>(g.n, w.B, g.root, w.word, w.ord);
    return cudaGetLastError();
}

cudaError_t launch_wilson(const GraphView &g, WaveView w, uint64_t seed, const int64_t *sids,
                          int64_t step_cap, cudaStream_t s) {
    k_wilson<<<(unsigned)((w.B + 127) / 128), 128, 0, s>>>(g, w, seed, sids, step_cap);
    return cudaGetLastError();
}

}  // namespace kc
