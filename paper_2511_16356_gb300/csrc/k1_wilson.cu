// Wilson's loop-erased-walk sampler (Sec. 2.2; Algorithm 1, "wilson(G, r)").
//
// Two walkers.  k_wilson_warp (the default) runs 32 concurrent walkers of one
// tree per warp (described below).  k_wilson runs one tree per lane as a flat
// state machine (SEEK a start vertex outside the tree, WALK, count the
// loop-erased path, commit it); every iteration does its phase's arithmetic,
// then one gather, then the phase's resolution, so lanes in different phases
// share one memory round trip.  Both can be chained (the lane walker stops at a
// start boundary and the warp walker resumes the tree).  The departure of u on
// its k-th visit follows neighbour bounded(seed, u, k, sample, WALK, deg u): in
// the lane walker loop erasure is implicit (next[u] is overwritten on the next
// departure), and by cycle popping the tree and step count depend neither on
// the start order nor on the walker.
//
// Per step a walker touches one 32-byte vertex record (degree, offset and the
// first neighbours) and the 8-byte walker word of the next vertex; both loads
// are issued together.  Committing a path of length L writes the words with
// the in-tree flag and depth and the path, parent first, into `ord`.
#include <algorithm>

#include "kc_common.cuh"

namespace kc {

namespace {

enum : int { kSeek = 0, kWalk = 1, kCount = 2, kCommit = 3 };

__global__ void k_wave_init(int64_t n, int64_t B, int32_t root, uint64_t *word, int32_t *ord) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= B) return;
    word[t * n + root] = w_make(-1, 0, true);
    ord[t * n] = root;
}

// Starts are taken in the order sorder[0 .. n) (id order when sorder is null).
// With rs_q set the lane may stop early, at a start boundary -- no walk in
// flight, every vertex either in the tree or free with its departure count --
// when it reaches order index q_stop, or when `done` (trees of the wave that
// already finished) has reached stop_at.  It then saves the order index of its
// next start and its order position in rs_q / rs_pos (rs_q = -1 for a
// finished tree), and the 32-walker kernel resumes the tree from there.
// kReject: step_cap bounds the tree's departures and a tree that exceeds it is
// abandoned (steps = -1) instead of failing the wave -- rejection by walk
// length.  With done_flag set, each lane publishes its finished tree to the
// host (depth + 1, or -1 when rejected) for the pipelined traversal.
// One-warp blocks: a wave of ten thousand lanes is ~300 warps, fewer than the
// SMs' schedulers, so each warp runs alone on its scheduler, latency-bound;
// one-warp blocks spread the warps over every SM (and its L1).
constexpr int kLaneWalkerBlock = 32;
template <bool kReject>
__global__ void __launch_bounds__(kLaneWalkerBlock) k_wilson(GraphView g, WaveView w, uint64_t seed,
                                                const int64_t *__restrict__ sids,
                                                const int32_t *__restrict__ sorder,
                                                int64_t step_cap, int32_t *rs_q, int32_t *rs_pos,
                                                unsigned int *done, int64_t q_stop,
                                                int64_t stop_at, volatile int32_t *done_flag) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= w.B) return;
    const int64_t n = g.n;
    uint64_t *__restrict__ word = w.word + t * n;
    int32_t *__restrict__ ord = w.ord + t * n;
    const VRec *__restrict__ rec = g.rec;
    const uint32_t sample = (uint32_t)sids[t];
    const PhiloxKeys keys = philox_keys(seed);

    int64_t steps = 0;
    int32_t pos = w.pos0;  // ord[0 .. pos0) already placed (the root, or an edge)
    int32_t q = 0;         // order index of the current start
    int32_t s = 0;         // current start vertex
    int32_t u = 0;         // walker position (WALK) / path cursor (COUNT, COMMIT)
    uint64_t wu = 0;       // word of u (WALK)
    VRec ru;               // record of u (WALK)
    ru.deg = 1;
    int32_t len = 0, i = 0, dh = 0, maxd = 0;
    int phase = kSeek;
    bool stopped = false;
    bool rejected = false;

    // Every iteration: phase-specific arithmetic, then ONE gather (the word of
    // one vertex, with its record when the lane may walk from it), then
    // phase-specific resolution.  Lanes of a warp sit in different phases, so
    // a gather per phase branch would serialise up to four memory round trips.
    for (;;) {
        int32_t a;
        bool want_rec = true;
        if (phase == kWalk) {
            const uint32_t k = bounded_draw_k(keys, seed, (uint32_t)u, w_count(wu), sample,
                                              kTagWalk, (uint32_t)ru.deg);
            int32_t v;
            if (k < (uint32_t)kInline) {
                // register select instead of a dynamic index into the record
                v = ru.nbr[0];
#pragma unroll
                for (int z = 1; z < kInline; ++z) v = (k == (uint32_t)z) ? ru.nbr[z] : v;
            } else {
                const uint64_t off = (uint64_t)ru.off_lo | ((uint64_t)ru.off_hi << 32);
                v = g.col[off + k];
            }
            word[u] = w_make(v, w_count(wu) + 1, false);
            if (kReject && ++steps > step_cap) {
                rejected = true;
                break;
            }
            if ((!kReject && ++steps > step_cap) || w_count(wu) + 1 >= (1u << 25)) {
                atomicOr(w.err, kErrStepLimit);
                break;
            }
            a = v;
        } else if (phase == kSeek) {
            if (q >= n) break;
            if (rs_q && (q >= q_stop || ((q & 255) == 0 && stop_at > 0 &&
                                         (int64_t)*(volatile unsigned int *)done >= stop_at))) {
                stopped = true;
                break;
            }
            s = sorder ? sorder[q] : q;
            a = s;
        } else {  // kCount, kCommit: the path cursor
            a = u;
            want_rec = false;
        }
        const uint64_t wa = word[a];
        VRec ra;
        ra.deg = 1;
        if (want_rec) ra = load_rec(rec + a);

        if (phase == kWalk) {
            if (w_in_tree(wa)) {
                u = s;
                len = 0;
                phase = kCount;
            } else {
                u = a;
                wu = wa;
                ru = ra;
            }
        } else if (phase == kSeek) {
            if (w_in_tree(wa)) {
                ++q;
            } else {
                u = s;
                wu = wa;
                ru = ra;
                phase = kWalk;
            }
        } else if (phase == kCount) {
            // length of the loop-erased path from s and the depth of its tree end
            if (w_in_tree(wa)) {
                dh = (int32_t)w_count(wa);
                u = s;
                i = 0;
                phase = kCommit;
            } else {
                ++len;
                u = w_next(wa);
                if (len > n || u < 0 || u >= n) {  // a path longer than n means corrupt state
                    atomicOr(w.err, kErrBadTree);
                    break;
                }
            }
        } else {  // kCommit
            const int32_t nx = w_next(wa);
            const int32_t d = dh + len - i;
            word[u] = w_make(nx, (uint32_t)d, true);
            ord[pos + len - 1 - i] = u;
            if (d > maxd) maxd = d;
            ++i;
            u = nx;
            if (i == len) {
                pos += len;
                ++q;
                phase = kSeek;
            }
        }
    }
    if (kReject && rejected) {
        w.steps[t] = -1;
        if (done_flag) {
            __threadfence_system();
            done_flag[t] = -1;  // finished, rejected
        }
        return;
    }
    w.steps[t] = steps;
    atomicMax(w.maxdepth, maxd);
    if (rs_q) {
        rs_q[t] = stopped ? q : -1;
        rs_pos[t] = pos;
        if (!stopped) atomicAdd(done, 1u);
    }
    if (done_flag) {
        // publish the finished tree (its depth + 1) after its words and order
        __threadfence_system();
        done_flag[t] = maxd + 1;
    }
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
// every 4th iteration by pointer doubling over shuffles.  No lane ever spins on
// another warp.
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
// Plain (L1-cached) accesses: the words of a tree are shared by the lanes of
// one warp only, and __syncwarp orders their stores before the next loads.
__device__ __forceinline__ uint64_t ld_word(const uint64_t *p) { return *p; }
__device__ __forceinline__ void st_word(uint64_t *p, uint64_t v) { *p = v; }

enum : int {
    pIdle = 0,     // needs a start vertex
    pWalk = 1,     // owns frontier c and departs from it
    pWait = 2,     // arrow (or empty path) points at x, owned by another lane
    pPopSet = 4,   // read the re-departure vertex before freeing a popped segment
    pPop = 5,      // free the vertices pcur .. pend of a popped cycle
    pCount = 6,    // length of the committed path
    pCommit = 7,   // write in-tree words, depths and the parent-first order
    pDone = 8
};

// With rs_q set, warp t resumes wave tree t where k_wilson stopped it: at order
// index rs_q[t] of the same start order and order position rs_pos[t], adding
// to its step count (rs_q[t] < 0: the tree is finished and the warp exits).
// Otherwise warp t samples tree t from scratch.
// One warp per block: a block frees its SM slot as soon as its own tree is
// done (tree times vary several-fold on long-diameter graphs, and a 4-warp
// block would hold three finished warps' registers until its slowest tree).
// kMulti: block j walks tree mw.entry[j].y of graph mw.entry[j].x, every graph
// with its own view, wave, seed, sample ids, start order and step cap (the
// batched multi-graph launch); otherwise one graph and wave as passed.
// kReject: step_cap bounds the tree's total departures (the warp's sum), and a
// tree that exceeds it is abandoned and marked steps = -1 instead of failing the
// wave (rejection by walk length, which keeps the accepted trees uniform).
constexpr int kWarpWalkerBlock = 32;
template <bool kMulti, bool kReject>
__global__ void __launch_bounds__(kWarpWalkerBlock, 24)
    k_wilson_warp(GraphView g_in, WaveView w_in, uint64_t seed_in,
                  const int64_t *__restrict__ sids_in, const int32_t *__restrict__ sorder_in,
                  int64_t step_cap_in, int64_t iter_cap_in, const int32_t *__restrict__ rs_q,
                  const int32_t *__restrict__ rs_pos, volatile int32_t *done_flag, MultiWalk mw) {
    const unsigned kFull = 0xFFFFFFFFu;
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    __shared__ int32_t xs[32];  // vertex each cycle lane's predecessor waits on
    GraphView g;
    WaveView w;
    uint64_t seed;
    const int64_t *sids;
    const int32_t *sorder;
    int64_t step_cap, iter_cap, t;
    if constexpr (kMulti) {
        if ((int64_t)blockIdx.x >= mw.count) return;
        const int2 e = mw.entry[blockIdx.x];
        g = mw.graphs[e.x];
        w = mw.waves[e.x];
        seed = mw.seeds[e.x];
        sids = mw.sids[e.x];
        sorder = mw.sorders[e.x];
        step_cap = mw.step_caps[e.x];
        iter_cap = 4 * step_cap + 64 * g.n + 4096;
        t = e.y;
    } else {
        g = g_in;
        w = w_in;
        seed = seed_in;
        sids = sids_in;
        sorder = sorder_in;
        step_cap = step_cap_in;
        iter_cap = iter_cap_in;
        t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
        if (t >= w.B) return;               // whole warp
        if (rs_q && rs_q[t] < 0) return;    // whole warp: finished by the lane walker
    }
    const int64_t n = g.n;
    uint64_t *word = w.word + t * n;
    int32_t *ord = w.ord + t * n;
    const VRec *__restrict__ rec = g.rec;
    const uint32_t sample = (uint32_t)sids[t];
    const PhiloxKeys keys = philox_keys(seed);

    int ph = pIdle;
    bool has_path = false;
    int32_t s = -1, c = -1, x = -1, u = -1, pcur = -1, pend = -1, prew = -1;
    uint32_t cc = 0;
    VRec rc;
    rc.deg = 1;
    int32_t len = 0, i = 0, dh = 0, mypos = 0, maxd = 0;
    int64_t steps = 0;
    int64_t next_start = rs_q ? (int64_t)rs_q[t] : 0;  // warp-uniform
    int64_t pos = rs_q ? (int64_t)rs_pos[t] : w.pos0;   // warp-uniform, ord[0 .. pos) placed
    bool bad = false;
    bool rejected = false;  // warp-uniform

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
        // a lane that met a bad state stopped itself (pDone, nothing loaded);
        // the warp notices within 8 iterations
        if (it > iter_cap || ((it & 7) == 0 && __any_sync(kFull, bad))) {
            if (lane == 0) atomicOr(w.err, bad ? kErrBadTree : kErrIterLimit);
            break;
        }
        if constexpr (kReject) {
            // every 8th iteration: abandon the tree once its departures pass
            // the cap (the final count is checked again at the end)
            if ((it & 7) == 0) {
                long long tt = (long long)steps;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) tt += __shfl_xor_sync(kFull, tt, o);
                if (tt > step_cap) {
                    rejected = true;
                    break;
                }
            }
        }
        // ---- act: departures and the address each lane reads this iteration
        int32_t ld = -1;
        if (ph == pWalk) {
            const uint32_t k = bounded_draw_k(keys, seed, (uint32_t)c, cc, sample, kTagWalk,
                                              (uint32_t)rc.deg);
            const int32_t v = rec_neighbor(rc, g.col, k);
            st_word(word + c, o_own(v, cc + 1, lane));
            cc += 1;
            ++steps;
            x = v;
            ld = v;
            if (cc >= kCountMask || (!kReject && steps > step_cap)) {
                atomicOr(w.err, kErrStepLimit);
                bad = true;
                ph = pDone;
                ld = -1;
            }
        } else if (ph == pIdle) {
            ld = s;
        } else if (ph == pWait) {
            ld = x;
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
        if ((may_walk || ph == pPopSet) && ld >= 0) rl = rec[ld];
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
                // loop closed on the own path: free next(ld) .. c, then re-depart
                // from ld, whose departure count and record are kept meanwhile
                prew = ld;
                cc = o_count(wl);
                rc = rl;
                pcur = w_next(wl);
                pend = c;
                ph = pPop;
            } else {
                if (ph == pIdle) has_path = false;
                x = ld;
                ph = pWait;
            }
        } else if (ph == pPopSet) {
            cc = o_count(wl);
            rc = rl;
            if (prew == c) {
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
                ph = pWalk;
            } else {
                pcur = nx;
                if (pcur < 0 || pcur >= n) {
                    bad = true;
                    ph = pDone;
                }
            }
        } else if (ph == pCount) {
            if (inT) {
                dh = (int32_t)w_count(wl);
                fin = true;
            } else {
                ++len;
                u = w_next(wl);
                if (len > n || u < 0 || u >= n) {
                    bad = true;
                    ph = pDone;
                }
            }
        } else if (ph == pCommit) {
            const int32_t nx = w_next(wl);
            const int32_t d = dh + len - i;
            st_word(word + u, w_make(nx, (uint32_t)d, true));
            const int64_t slot = (int64_t)mypos + len - 1 - i;
            if (slot > 0 && slot < n) ord[slot] = u;
            if (d > maxd) maxd = d;
            ++i;
            u = nx;
            if (i == len) ph = pIdle;
            if (slot <= 0 || slot >= n) {
                bad = true;
                ph = pDone;
            }
        }
        // ---- reserve slots of the parent-first order for paths that reached the tree
        if (__any_sync(kFull, fin)) {
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
        // ---- wait cycles: each lane that stays waiting points at the owner of its
        // target.  A lane lies on a cycle of this functional graph exactly when it
        // is succ^32 of some lane (a 32-step path among 32 lanes must have entered
        // a cycle, and succ^32 permutes each cycle), found by 5 doubling rounds.
        const int succ = (was_wait && ph == pWait && has_path && own && ownr != lane) ? ownr : -1;
        // (a cycle of waits persists until popped, so every 4th iteration suffices)
        if ((it & 3) == 0 && __popc(__ballot_sync(kFull, succ >= 0)) >= 2) {
            int z = succ;
#pragma unroll
            for (int r = 0; r < 5; ++r) {
                const int zz = __shfl_sync(kFull, z, z < 0 ? lane : z);
                z = z < 0 ? -1 : zz;
            }
            const unsigned onm = __reduce_or_sync(kFull, z >= 0 ? 1u << z : 0u);
            if (onm) {
                // each lane on a cycle hands the vertex it waits on to its successor,
                // whose path contains it: that lane pops the cycle segment after the
                // vertex and re-departs from it
                const bool on = (onm >> lane) & 1u;
                if (on) xs[succ] = x;
                __syncwarp();
                if (on) {
                    prew = xs[lane];
                    ph = pPopSet;
                }
                __syncwarp();
            }
        }
    }
    if constexpr (kReject) {
        if (rejected) {
            if (lane == 0) {
                w.steps[t] = -1;
                if (done_flag) {
                    __threadfence_system();
                    done_flag[t] = -1;  // finished, rejected
                }
            }
            return;
        }
    }
    long long tot = (long long)steps;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) tot += __shfl_down_sync(kFull, tot, o);
    int md = maxd;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) md = max(md, __shfl_down_sync(kFull, md, o));
    const bool over = kReject && __shfl_sync(kFull, tot, 0) > step_cap;
    if (lane == 0) {
        if (over) {
            w.steps[t] = -1;  // finished between two checks, but past the cap
        } else {
            w.steps[t] = (rs_q ? w.steps[t] : 0) + tot;
            atomicMax(w.maxdepth, md);
        }
    }
    if (done_flag && over) {
        if (lane == 0) {
            __threadfence_system();
            done_flag[t] = -1;  // finished, rejected
        }
        return;
    }
    if (done_flag) {
        // publish the finished tree (its depth + 1) to the host, after every
        // lane's words and order entries are visible
        __threadfence_system();
        __syncwarp();
        if (lane == 0) {
            __threadfence_system();
            done_flag[t] = md + 1;
        }
    }
}

}  // namespace

cudaError_t launch_wilson_warp(const GraphView &g, WaveView w, uint64_t seed, const int64_t *sids,
                               const int32_t *sorder, int64_t step_cap, cudaStream_t s,
                               const int32_t *rs_q, const int32_t *rs_pos, int32_t *done_flag) {
    // a correct run needs at most about 3 iterations per departure (walk,
    // count, commit / pop), however the walkers serialise
    const int64_t iter_cap = 4 * step_cap + 64 * g.n + 4096;
    k_wilson_warp<false, false><<<(unsigned)w.B, kWarpWalkerBlock, 0, s>>>(
        g, w, seed, sids, sorder, step_cap, iter_cap, rs_q, rs_pos, done_flag, MultiWalk{});
    return cudaGetLastError();
}

cudaError_t launch_wilson_warp_reject(const GraphView &g, WaveView w, uint64_t seed,
                                      const int64_t *sids, const int32_t *sorder,
                                      int64_t tree_cap, cudaStream_t s, int32_t *done_flag) {
    // tree_cap bounds the whole tree's departures, and an iteration may move
    // as little as one lane: a generous bound that no accepted tree reaches
    const int64_t iter_cap = 16 * std::min<int64_t>(tree_cap, (int64_t)1 << 40) + 64 * g.n + 4096;
    k_wilson_warp<false, true><<<(unsigned)w.B, kWarpWalkerBlock, 0, s>>>(
        g, w, seed, sids, sorder, tree_cap, iter_cap, nullptr, nullptr, done_flag, MultiWalk{});
    return cudaGetLastError();
}

int wilson_warp_blocks_per_sm() {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_wilson_warp<false, false>, kWarpWalkerBlock,
                                                      0) != cudaSuccess) {
        (void)cudaGetLastError();
        return 0;
    }
    return b;
}

cudaError_t launch_wilson_warp_multi(const MultiWalk &mw, cudaStream_t s) {
    if (mw.count <= 0) return cudaSuccess;
    k_wilson_warp<true, false><<<(unsigned)mw.count, kWarpWalkerBlock, 0, s>>>(
        GraphView{}, WaveView{}, 0, nullptr, nullptr, 0, 0, nullptr, nullptr, nullptr, mw);
    return cudaGetLastError();
}

cudaError_t launch_wave_init(const GraphView &g, WaveView w, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(w.word, 0, sizeof(uint64_t) * (size_t)(w.B * g.n), s);
    if (e != cudaSuccess) return e;
    k_wave_init<<<(unsigned)((w.B + 127) / 128), 128, 0, s>>>(g.n, w.B, g.root, w.word, w.ord);
    return cudaGetLastError();
}

cudaError_t launch_wilson(const GraphView &g, WaveView w, uint64_t seed, const int64_t *sids,
                          int64_t step_cap, cudaStream_t s, const int32_t *sorder, int32_t *rs_q,
                          int32_t *rs_pos, unsigned int *done, int64_t q_stop, int64_t stop_at,
                          int32_t *done_flag) {
    k_wilson<false><<<(unsigned)((w.B + kLaneWalkerBlock - 1) / kLaneWalkerBlock),
                      kLaneWalkerBlock, 0, s>>>(g, w, seed, sids, sorder, step_cap, rs_q, rs_pos,
                                                done, q_stop, stop_at, done_flag);
    return cudaGetLastError();
}

cudaError_t launch_wilson_reject(const GraphView &g, WaveView w, uint64_t seed,
                                 const int64_t *sids, const int32_t *sorder, int64_t tree_cap,
                                 cudaStream_t s, int32_t *done_flag) {
    k_wilson<true><<<(unsigned)((w.B + kLaneWalkerBlock - 1) / kLaneWalkerBlock),
                     kLaneWalkerBlock, 0, s>>>(g, w, seed, sids, sorder, tree_cap, nullptr, nullptr,
                                               nullptr, 0, 0, done_flag);
    return cudaGetLastError();
}

}  // namespace kc
