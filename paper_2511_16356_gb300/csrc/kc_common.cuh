// Internal declarations shared by the CUDA translation units of libkc.
// Layout of every device array is documented where it is declared.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/kc.h"

namespace kc {

// ---------------------------------------------------------------------------
// Random-number contract: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11),
// key = (seed lo, seed hi), counter = (c0, c1, c2, tag << 24 | retry), and
// Lemire's multiply-and-reject bounded integers over the block's four words.
// ---------------------------------------------------------------------------
constexpr uint32_t kPhiloxM0 = 0xD2511F53u;
constexpr uint32_t kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u;
constexpr uint32_t kPhiloxW1 = 0xBB67AE85u;

constexpr uint32_t kTagWalk = 0u;     // Wilson departures: (u, k, sample id)
constexpr uint32_t kTagSelect = 1u;   // update: choice of trees to replace / transform
constexpr uint32_t kTagLinkCut = 2u;  // ISM insert: edge of the cycle to cut
constexpr uint32_t kTagCutLink = 3u;  // ISM delete: crossing edge to link

__device__ __forceinline__ void philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                              uint32_t k0, uint32_t k1, uint32_t out[4]) {
#pragma unroll
    for (int i = 0; i < 10; ++i) {
        const uint32_t lo0 = kPhiloxM0 * c0;
        const uint32_t hi0 = __umulhi(kPhiloxM0, c0);
        const uint32_t lo1 = kPhiloxM1 * c2;
        const uint32_t hi1 = __umulhi(kPhiloxM1, c2);
        c0 = hi1 ^ c1 ^ k0;
        c1 = lo1;
        c2 = hi0 ^ c3 ^ k1;
        c3 = lo0;
        k0 += kPhiloxW0;
        k1 += kPhiloxW1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

// The ten round keys of a Philox4x32-10 key: the key schedule adds the Weyl
// constants once per round and depends on the seed only, so a walker computes
// it once and its draws skip the twenty additions.
struct PhiloxKeys {
    uint32_t k0[10], k1[10];
};
__device__ __forceinline__ PhiloxKeys philox_keys(uint64_t seed) {
    PhiloxKeys K;
    uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
#pragma unroll
    for (int i = 0; i < 10; ++i) {
        K.k0[i] = k0;
        K.k1[i] = k1;
        k0 += kPhiloxW0;
        k1 += kPhiloxW1;
    }
    return K;
}
// philox4x32_10 with the round keys precomputed
__device__ __forceinline__ void philox4x32_10_k(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                                const PhiloxKeys &K, uint32_t out[4]) {
#pragma unroll
    for (int i = 0; i < 10; ++i) {
        const uint32_t lo0 = kPhiloxM0 * c0;
        const uint32_t hi0 = __umulhi(kPhiloxM0, c0);
        const uint32_t lo1 = kPhiloxM1 * c2;
        const uint32_t hi1 = __umulhi(kPhiloxM1, c2);
        c0 = hi1 ^ c1 ^ K.k0[i];
        c1 = lo1;
        c2 = hi0 ^ c3 ^ K.k1[i];
        c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

// Uniform integer in [0, s), s >= 1: all four words and the retry counter.
static __device__ __noinline__ uint32_t bounded_draw_full(uint64_t seed, uint32_t c0, uint32_t c1,
                                                   uint32_t c2, uint32_t tag, uint32_t s) {
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    for (uint32_t retry = 0; retry < (1u << 24); ++retry) {
        uint32_t w[4];
        philox4x32_10(c0, c1, c2, (tag << 24) | retry, k0, k1, w);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const uint64_t m = (uint64_t)w[j] * (uint64_t)s;
            const uint32_t low = (uint32_t)m;
            if (low < s) {  // only then can the rejection threshold matter
                const uint32_t thr = (0u - s) % s;
                if (low < thr) continue;
            }
            return (uint32_t)(m >> 32);
        }
    }
    return 0;
}

// Same result as bounded_draw_full.  Fast path: word 0 of the first block is
// accepted outright when the low half of x*s is >= s (the rejection threshold
// (2^32 - s) mod s is below s), which fails with probability s / 2^32.
__device__ __forceinline__ uint32_t bounded_draw(uint64_t seed, uint32_t c0, uint32_t c1,
                                                 uint32_t c2, uint32_t tag, uint32_t s) {
    uint32_t w[4];
    philox4x32_10(c0, c1, c2, tag << 24, (uint32_t)seed, (uint32_t)(seed >> 32), w);
    const uint64_t m = (uint64_t)w[0] * (uint64_t)s;
    if (__builtin_expect((uint32_t)m >= s, 1)) return (uint32_t)(m >> 32);
    return bounded_draw_full(seed, c0, c1, c2, tag, s);
}

// bounded_draw with precomputed round keys (same result)
__device__ __forceinline__ uint32_t bounded_draw_k(const PhiloxKeys &K, uint64_t seed, uint32_t c0,
                                                   uint32_t c1, uint32_t c2, uint32_t tag,
                                                   uint32_t s) {
    uint32_t w[4];
    philox4x32_10_k(c0, c1, c2, tag << 24, K, w);
    const uint64_t m = (uint64_t)w[0] * (uint64_t)s;
    if (__builtin_expect((uint32_t)m >= s, 1)) return (uint32_t)(m >> 32);
    return bounded_draw_full(seed, c0, c1, c2, tag, s);
}

// ---------------------------------------------------------------------------
// Vertex record used by the walk: one 32-byte sector per vertex holding the
// degree, the CSR offset and the first kInline neighbours, so a step on a
// vertex of degree <= kInline costs one sector of graph data.
// ---------------------------------------------------------------------------
constexpr int kInline = 5;
struct __align__(32) VRec {
    int32_t deg;
    uint32_t off_lo;
    uint32_t off_hi;
    int32_t nbr[kInline];
};
static_assert(sizeof(VRec) == 32, "VRec must be one sector");

// the record as two 16-byte loads through the read-only data path
__device__ __forceinline__ VRec load_rec(const VRec *p) {
    const uint4 *q = reinterpret_cast<const uint4 *>(p);
    const uint4 a = __ldg(q), b = __ldg(q + 1);
    VRec r;
    r.deg = (int32_t)a.x;
    r.off_lo = a.y;
    r.off_hi = a.z;
    r.nbr[0] = (int32_t)a.w;
    r.nbr[1] = (int32_t)b.x;
    r.nbr[2] = (int32_t)b.y;
    r.nbr[3] = (int32_t)b.z;
    r.nbr[4] = (int32_t)b.w;
    return r;
}

// ---------------------------------------------------------------------------
// Per-tree vertex word of the walker (8 bytes):
//   bits  0..31  next / parent (int32; -1 for the root)
//   bits 32..62  departure count while the vertex is outside the tree,
//                depth once it is in the tree
//   bit  63      in-tree flag
// ---------------------------------------------------------------------------
constexpr uint64_t kInTree = 1ull << 63;
__host__ __device__ __forceinline__ int32_t w_next(uint64_t w) { return (int32_t)(uint32_t)w; }
__host__ __device__ __forceinline__ uint32_t w_count(uint64_t w) {
    return (uint32_t)(w >> 32) & 0x7FFFFFFFu;
}
__host__ __device__ __forceinline__ bool w_in_tree(uint64_t w) { return (w & kInTree) != 0; }
__host__ __device__ __forceinline__ uint64_t w_make(int32_t next, uint32_t count, bool in_tree) {
    return (uint64_t)(uint32_t)next | ((uint64_t)(count & 0x7FFFFFFFu) << 32) |
           (in_tree ? kInTree : 0ull);
}

// Error word bits written by kernels (read back by the host after a phase).
constexpr uint32_t kErrStepLimit = 1u;
constexpr uint32_t kErrBadTree = 2u;
constexpr uint32_t kErrIterLimit = 4u;

// ---------------------------------------------------------------------------
// Device views
// ---------------------------------------------------------------------------
struct GraphView {
    int64_t n;
    int64_t twom;
    const int64_t *row_off;  // [n+1]
    const int32_t *col;      // [2m]
    const int32_t *deg;      // [n]
    const VRec *rec;         // [n]
    int32_t root;
    int32_t ecc;
    const int32_t *p0;       // [n] tau0 parent, -1 at the root
    const int32_t *in0;      // [n] tau0 DFN
    const int32_t *out0;     // [n]
};

// Workspace of one wave of B trees; every per-tree array is tree-major
// ([tree][vertex], tree stride = n).
struct WaveView {
    int64_t B;               // trees in this wave
    int64_t n;
    uint64_t *word;          // [B][n] walker words (parent + depth afterwards)
    int32_t *ord;            // [B][n] parent-first order from the walk (root first);
                             // reused as the DFS stack by the BIT variant
    int32_t *size;           // [B][n] subtree sizes
    int64_t *vol;            // [B][n] subtree volumes
    int32_t *din;            // [B][n] DFN (sibling offsets before the top-down pass)
    int32_t *aux;            // [B][n] per-parent running sums, then preorder (BIT variant)
    int64_t *bit;            // [B][n+1] Fenwick array (BIT variant), may be null
    int64_t *steps;          // [B]
    int64_t *f;              // [B]
    uint32_t *err;           // [1] error bits (kErr*)
    int32_t *maxdepth;       // [1] largest tree depth seen in the wave
    int32_t *stack;          // [B][stack_cap] x 4 int32 DFS stack (BIT variant)
    int64_t stack_cap;       // entries per tree
    int32_t pos0 = 1;        // vertices already placed in ord before the walk
    const int32_t *tmap = nullptr;  // sub-wave tree t -> wave tree tmap[t] (word, ord, f,
                                    // steps); null: the identity
};

// One preorder segment of a tree for the segmented BIT evaluation of f: its
// Fenwick array (`bit` is the 1-based base, entries 1 .. n used), its stack
// (stack_cap int4 entries) and the positions [lo, hi) of sub-wave tree t.
struct TtfSeg {
    int64_t *bit;
    int4 *stk;
    int32_t t, lo, hi, pad;
};

// wave tree of sub-wave tree t
__host__ __device__ __forceinline__ int64_t wave_tree(const WaveView &w, int64_t t) {
    return w.tmap ? (int64_t)w.tmap[t] : t;
}

// ---------------------------------------------------------------------------
// Host handle
// ---------------------------------------------------------------------------
struct PhaseTimer {
    double ms = 0.0;
    int64_t launches = 0;
};

// A captured chunk of conjugate-gradient iterations (k8_resistance.cu) and the
// pointers and size it was captured for.
struct CgGraph {
    cudaGraphExec_t exec = nullptr;
    const void *key[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    int launches = 0;  // kernel launches one replay stands for
    cudaStream_t capture_stream = nullptr;
};

}  // namespace kc

struct kc_graph {
    kc_config cfg;
    int device = 0;
    cudaStream_t stream = nullptr;
    int64_t n = 0, m = 0;
    // device graph
    int64_t *d_row_off = nullptr;
    int32_t *d_col = nullptr;
    int32_t *d_deg = nullptr;
    kc::VRec *d_rec = nullptr;
    int32_t root = -1, ecc = 0;
    int32_t *d_p0 = nullptr, *d_level0 = nullptr, *d_in0 = nullptr, *d_out0 = nullptr;
    int32_t ttf_variant = KC_TTF_SCAN;
    int32_t walker = KC_WALK_WARP;
    // host copy of the graph (validated CSR, needed by updates)
    std::vector<int64_t> h_row_off;
    std::vector<int32_t> h_col;
    // pool
    bool seeded = false;
    uint64_t seed = 0;
    int64_t pool = 0, pool_cap = 0;
    int64_t next_sid = 0;
    int64_t ws_limit = 0;  // workspace byte budget (0: a share of free memory)
    int trav_mode = -1;     // kTrav* for f, -1: chosen from the graph
    bool tuning = false;    // pilot waves of the autotuner (no pipelining)
    bool tuned = false;
    double tune_ms[4] = {0, 0, 0, 0};
    int64_t resident_trees = 0;  // trees the 32-walker kernel runs at once on the device
    int64_t num_sms = 0;
    int64_t *d_f = nullptr;
    double *d_w = nullptr;
    int64_t *d_steps = nullptr;
    int64_t *d_sid = nullptr;
    int32_t *d_parents = nullptr;  // [pool_cap][n] when keep_trees
    std::vector<uint8_t> h_modified; // tree changed by an update (not reproducible from its id)
    // workspace
    void *d_ws = nullptr;
    size_t ws_bytes = 0;
    int32_t *d_stack = nullptr;     // BIT-variant DFS stacks, [trees][cap] x int4
    size_t stack_bytes = 0;
    int32_t *d_sorder = nullptr;    // start order of the concurrent walkers
    void *d_ub = nullptr;           // update buffers: slots, factors, selection, flags
    size_t ub_bytes = 0;
    size_t col_cap = 0;             // capacity of d_col (entries)
    int32_t *d_edit = nullptr;      // scratch column array of a graph edit
    size_t edit_cap = 0;
    double *d_cg = nullptr;         // conjugate-gradient vectors of R(u, v)
    kc::CgGraph cg_graph;           // their captured iteration chunk
    bool host_csr_stale = false;    // h_row_off / h_col behind the device CSR
    int64_t ws_trees = 0;
    uint32_t *d_err = nullptr;
    void *d_scratch = nullptr;      // small reduction scratch
    size_t scratch_bytes = 0;
    int64_t last_wave = 0;
    int64_t total_steps = 0;
    int64_t updates_applied = 0, trees_resampled = 0;
    int64_t trees_rejected = 0;  // abandoned by rejection by walk length
    int64_t rej_drawn = 0, rej_accepted = 0;  // trees walked / accepted under rejection
    int64_t update_seq = 0;
    double last_r = 0.0;
    int64_t last_cg_iters = 0;
    kc::PhaseTimer t_wilson, t_traverse, t_ttf, t_reduce, t_update, t_setup, t_init;
    double ms_upd_part[4] = {0, 0, 0, 0};  // kc_update: graph edit, R, trees, refresh
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    // pipelined waves: a second stream for traversal/TTF chunks, host-mapped
    // per-tree completion flags written by the walker, the chunks' tree maps
    cudaStream_t stream2 = nullptr;
    int32_t *h_done = nullptr, *d_done = nullptr;  // mapped pinned host memory
    int32_t *h_map = nullptr;                      // pinned staging of tree maps
    // segmented BIT evaluation: segment tables of the current wave (pinned
    // staging and device copy, seg_used entries taken), and the handle buffer
    // for segments that free memory does not hold (cfg.ttf_segments >= 2)
    kc::TtfSeg *h_segtab = nullptr, *d_segtab = nullptr;
    int64_t segtab_cap = 0, seg_used = 0;
    char *d_segx = nullptr;
    size_t segx_bytes = 0;
    int32_t *d_map = nullptr;
    int64_t done_cap = 0;
    std::string last_error;
};

namespace kc {

// Launch helpers implemented in the .cu files.  Each returns cudaGetLastError().
cudaError_t launch_build_records(const GraphView &g, VRec *rec, int32_t *deg, cudaStream_t s);
cudaError_t launch_validate(const GraphView &g, uint32_t *flags, cudaStream_t s);
cudaError_t launch_root(const GraphView &g, unsigned long long *best, cudaStream_t s);
cudaError_t launch_bfs_init(int64_t n, int32_t r, int32_t *level, cudaStream_t s);
cudaError_t launch_dfs_tree(const GraphView &g, int32_t r, int32_t *p0, int32_t *level,
                            int32_t *sv, int64_t *se, int32_t *deepest, int32_t *unreached,
                            cudaStream_t s);
cudaError_t launch_tau0_from_words(int64_t n, const uint64_t *word, int32_t *p0, int32_t *level,
                                   int32_t *deepest, int32_t *outside, cudaStream_t s);
cudaError_t launch_argmax_score(int64_t n, const int32_t *la, const int32_t *lb, int mode,
                                unsigned long long *best, cudaStream_t s);
cudaError_t launch_central_pick(int64_t n, const int32_t *deg, int32_t dmax, const int32_t *la,
                                const int32_t *lb, const int32_t *lc, unsigned long long *best,
                                int32_t *ties, cudaStream_t s);
cudaError_t launch_bfs_level(const GraphView &g, int32_t lev, int32_t *level, int32_t *changed,
                             cudaStream_t s);
cudaError_t launch_bfs_parent(const GraphView &g, const int32_t *level, int32_t *p0,
                              int32_t *unreached, cudaStream_t s);
cudaError_t launch_tau0_words(int64_t n, const int32_t *p0, const int32_t *level, uint64_t *word,
                              cudaStream_t s);
cudaError_t launch_level_order(int64_t n, int32_t ecc, const int32_t *level, int32_t *hist,
                               int32_t *ord, cudaStream_t s);

cudaError_t launch_wave_init(const GraphView &g, WaveView w, cudaStream_t s);
// Batched multi-graph walk: device tables indexed by graph, one entry
// (graph, tree of its wave) per warp.
struct MultiWalk {
    const GraphView *graphs = nullptr;
    const WaveView *waves = nullptr;
    const uint64_t *seeds = nullptr;
    const int64_t *const *sids = nullptr;
    const int32_t *const *sorders = nullptr;
    const int64_t *step_caps = nullptr;
    const int2 *entry = nullptr;
    int64_t count = 0;
};
cudaError_t launch_wilson_warp_multi(const MultiWalk &mw, cudaStream_t s);
// resident one-warp blocks of the 32-walker kernel per SM (0 if the query fails)
int wilson_warp_blocks_per_sm();

// Batched multi-graph traversal / TTF: per-graph views and sub-wave buffers,
// one entry (graph, tree of its sub-wave) per warp (or per grid row).
struct MultiSub {
    const GraphView *graphs = nullptr;
    const WaveView *waves = nullptr;
    const int2 *entry = nullptr;
    int64_t count = 0;
};

// The tree a warp / grid row works on: table row `row` of a batched launch,
// or tree `row` of the single graph and wave passed by value.
template <bool kMulti>
__device__ __forceinline__ bool pick_tree(const MultiSub &ms, const GraphView &g_in,
                                          const WaveView &w_in, int64_t row, GraphView &g,
                                          WaveView &w, int64_t &t) {
    if constexpr (kMulti) {
        if (row >= ms.count) return false;
        const int2 e = ms.entry[row];
        g = ms.graphs[e.x];
        w = ms.waves[e.x];
        t = e.y;
        return true;
    } else {
        g = g_in;
        w = w_in;
        t = row;
        return t < w.B;
    }
}
// multi-graph chunked traversal (sizes, volumes, offsets, then DFN; preorder for
// waves with a BIT array) and TTF over tables built by the host; the caller
// zeroes each sub-wave's size and vol (and bit, f) first.  max_n: largest n.
cudaError_t launch_traverse_multi(const MultiSub &ms, cudaStream_t s);
cudaError_t launch_ttf_scan_multi(const MultiSub &ms, int64_t max_n, cudaStream_t s);
cudaError_t launch_ttf_bit_multi(const MultiSub &ms, cudaStream_t s);
cudaError_t launch_wilson(const GraphView &g, WaveView w, uint64_t seed, const int64_t *sids,
                          int64_t step_cap, cudaStream_t s, const int32_t *sorder = nullptr,
                          int32_t *rs_q = nullptr, int32_t *rs_pos = nullptr,
                          unsigned int *done = nullptr, int64_t q_stop = 0, int64_t stop_at = 0,
                          int32_t *done_flag = nullptr);
// one walker per tree with rejection by walk length (tree_cap departures): a
// rejected tree gets steps = -1 (and done flag -1) and no depth or order
cudaError_t launch_wilson_reject(const GraphView &g, WaveView w, uint64_t seed,
                                 const int64_t *sids, const int32_t *sorder, int64_t tree_cap,
                                 cudaStream_t s, int32_t *done_flag = nullptr);
cudaError_t launch_wilson_warp(const GraphView &g, WaveView w, uint64_t seed, const int64_t *sids,
                               const int32_t *sorder, int64_t step_cap, cudaStream_t s,
                               const int32_t *rs_q = nullptr, const int32_t *rs_pos = nullptr,
                               int32_t *done_flag = nullptr);
// 32 walkers per tree with rejection by walk length: a tree whose departures
// exceed tree_cap gets steps = -1 (and done flag -1) and no depth, order or
// finished words
cudaError_t launch_wilson_warp_reject(const GraphView &g, WaveView w, uint64_t seed,
                                      const int64_t *sids, const int32_t *sorder,
                                      int64_t tree_cap, cudaStream_t s,
                                      int32_t *done_flag = nullptr);
// Traversal modes: kTravCanonical numbers children in ascending id (the DFN the
// oracle reports and the update kernels enumerate by); the others give some
// valid DFN (enough for f): kTravChunked (warp per tree, for deep trees and
// small graphs) and kTravLeafUp (leaf-to-root atomics, for large shallow trees).
enum : int { kTravCanonical = 0, kTravChunked = 1, kTravLeafUp = 2 };
cudaError_t launch_traverse(const GraphView &g, WaveView w, bool want_preorder, cudaStream_t s,
                            int *launches = nullptr, int mode = kTravCanonical);
cudaError_t launch_ttf_scan(const GraphView &g, WaveView w, cudaStream_t s);
cudaError_t launch_ttf_bit(const GraphView &g, WaveView w, cudaStream_t s);
// f of the sub-wave's trees from segments that each start from the DFS state
// rebuilt at their first position; zeroes the segments' Fenwick arrays first and
// adds into w.f (zeroed by the caller).  segs: device table of nseg entries.
cudaError_t launch_ttf_bit_seg(const GraphView &g, WaveView w, const TtfSeg *segs, int64_t nseg,
                               cudaStream_t s);
cudaError_t launch_pool_append(WaveView w, int64_t first, int64_t *pool_f, double *pool_w,
                               int64_t *pool_steps, int64_t *pool_sid, const int64_t *sids,
                               int32_t *pool_parents, int64_t n, cudaStream_t s);
cudaError_t launch_pool_reduce(const int64_t *f, const double *w, int64_t count, int64_t twom,
                               void *scratch, cudaStream_t s);
cudaError_t launch_words_from_parents(int64_t n, int64_t B, const int32_t *parents,
                                      uint64_t *word, cudaStream_t s);

// Sample maintenance (k6_update.cu) and effective resistance (k8_resistance.cu).
cudaError_t launch_edge_pre_init(int64_t n, int64_t B, int32_t u, int32_t v, uint64_t *word,
                                 int32_t *ord, cudaStream_t s);
cudaError_t launch_words_to_slots(int64_t n, int64_t B, const uint64_t *word, const int64_t *slot,
                                  int32_t *pool_parents, int32_t r, int32_t top, uint32_t *err,
                                  cudaStream_t s);
cudaError_t launch_contains_edge(int64_t n, int64_t P, const int32_t *pool_parents, int32_t u,
                                 int32_t v, uint8_t *flag, cudaStream_t s);
cudaError_t launch_select(uint64_t seed, uint32_t seq, int64_t N, int64_t k, uint8_t *taken,
                          int64_t *out, cudaStream_t s);
cudaError_t launch_prepare_from_parents(int64_t n, int64_t B, int32_t root,
                                        const int32_t *pool_parents, const int64_t *slot,
                                        WaveView w, cudaStream_t s);
cudaError_t launch_link_cut(const int64_t *row_off, const int32_t *col, WaveView w,
                            const int64_t *slot, int32_t *pool_parents, double *factor, int32_t r,
                            int32_t u, int32_t v, uint64_t seed, uint32_t seq, bool insert,
                            cudaStream_t s);
cudaError_t launch_scale_slots(double *w, const int64_t *slot, const double *factor, int64_t B,
                               cudaStream_t s);
cudaError_t launch_weight_rescale(double *w, const uint8_t *flag, int64_t P, double *sums,
                                  double target_flagged, double target_rest, cudaStream_t s);
cudaError_t launch_weight_sums(const double *w, const uint8_t *flag, int64_t P, double *sums,
                               cudaStream_t s);
cudaError_t launch_scatter_results(const int64_t *slot, int64_t B, const int64_t *f,
                                   const int64_t *steps, const int64_t *sids, int64_t *pool_f,
                                   int64_t *pool_steps, int64_t *pool_sid, cudaStream_t s);
// R(u, v) = (e_u - e_v)^T L^+ (e_u - e_v) by Jacobi-preconditioned FP64 CG, in
// caller-owned scratch of cg_scratch_doubles(n) doubles.  With `cache`, the
// iterations between two residual checks run as one captured CUDA graph, kept
// in the cache for later calls on the same CSR, scratch and n.
void cg_graph_release(CgGraph &c);
size_t cg_scratch_doubles(int64_t n);
cudaError_t resistance_cg(const GraphView &g, int32_t u, int32_t v, double tol, int64_t max_iter,
                          double *scratch, double *R_out, int64_t *iters_out, int *launches,
                          cudaStream_t s, CgGraph *cache = nullptr);
// one edge insert / delete of the device CSR, rows kept sorted (k9_graph_edit.cu)
cudaError_t launch_csr_edit(int64_t n, int64_t twom, int64_t *row_off, int32_t *col,
                            int32_t *scratch, int64_t *pos, int32_t u, int32_t v, bool insert,
                            cudaStream_t s);

// Result layout of launch_pool_reduce in `scratch`.
struct PoolSums {
    long long f_hi;          // int128 sum of f as (hi, lo) limbs
    unsigned long long f_lo;
    double wf;               // sum w f / 2m
    double w;                // sum w
    double x2;               // sum (f / 2m)^2 (unit weights)
    long long count;
};

}  // namespace kc
