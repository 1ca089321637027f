// Host side of the C ABI declared in include/kc.h: handle lifetime, graph
// setup, wave planning for kc_sample (pipelined waves, batched multi-graph
// waves), the stopping rule of kc_estimate, sample maintenance, pool
// bookkeeping and the test hooks.  All arithmetic of the method runs in the
// kernels of the other translation units; this file only moves data, sizes
// launches and reads back scalars.
#include <cuda_runtime.h>

#include <algorithm>
#include <thread>
#include <chrono>
#include <array>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "kc_common.cuh"
#include "kc_host_graph.h"
#include "kc_host_stop.h"
#include "kc_host_plan.h"
#include "kc_host_seg.h"

namespace kc {
cudaError_t launch_out_from_size(int64_t n, const int32_t *din, const int32_t *size,
                                 int32_t *dout, cudaStream_t s);
cudaError_t launch_iota(int64_t *dst, int64_t start, int64_t count, cudaStream_t s);
}  // namespace kc

using namespace kc;

namespace {

struct Fail {
    kc_status st;
};

kc_status cuda_status(cudaError_t e) {
    return e == cudaErrorMemoryAllocation ? KC_ERR_OUT_OF_MEMORY : KC_ERR_CUDA;
}

#define KC_CK(g, expr)                                                       \
    do {                                                                     \
        cudaError_t _e = (expr);                                             \
        if (_e != cudaSuccess) {                                             \
            if (g) (g)->last_error = std::string(#expr) + ": " + cudaGetErrorString(_e); \
            (void)cudaGetLastError();                                        \
            throw Fail{cuda_status(_e)};                                     \
        }                                                                    \
    } while (0)

template <class T>
void dalloc(kc_graph *g, T **p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    KC_CK(g, cudaMalloc((void **)p, sizeof(T) * count));
}

template <class T>
void dfree(T *&p) {
    if (p && cudaFree((void *)p) != cudaSuccess) (void)cudaGetLastError();
    p = nullptr;
}

void hfree(void *p) {
    if (p && cudaFreeHost(p) != cudaSuccess) (void)cudaGetLastError();
}

// Launch checks read the runtime's per-thread last error, so an error that an
// earlier, unrelated runtime call left pending on the calling thread would be
// reported as this call's failure.  Entry points that do device work clear it
// first (a sticky error of a broken context still fails the next call).
void clear_stale_error() { (void)cudaGetLastError(); }

// A blocking copy ordered after the handle's stream: the legacy default stream
// does not wait for non-blocking streams, so plain cudaMemcpy could read
// results before the handle's kernels finish.
cudaError_t copy_sync(kc_graph *g, void *dst, const void *src, size_t bytes, cudaMemcpyKind kind) {
    cudaError_t e = cudaMemcpyAsync(dst, src, bytes, kind, g->stream);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(g->stream);
}

GraphView view_of(const kc_graph *g) {
    GraphView v;
    v.n = g->n;
    v.twom = 2 * g->m;
    v.row_off = g->d_row_off;
    v.col = g->d_col;
    v.deg = g->d_deg;
    v.rec = g->d_rec;
    v.root = g->root;
    v.ecc = g->ecc;
    v.p0 = g->d_p0;
    v.in0 = g->d_in0;
    v.out0 = g->d_out0;
    return v;
}

// Phase timing with CUDA events on the handle's stream.
struct Phase {
    kc_graph *g;
    PhaseTimer &t;
    Phase(kc_graph *g_, PhaseTimer &t_) : g(g_), t(t_) { KC_CK(g, cudaEventRecord(g->ev0, g->stream)); }
    void done(int launches) {
        KC_CK(g, cudaEventRecord(g->ev1, g->stream));
        KC_CK(g, cudaEventSynchronize(g->ev1));
        float ms = 0.f;
        KC_CK(g, cudaEventElapsedTime(&ms, g->ev0, g->ev1));
        t.ms += ms;
        t.launches += launches;
    }
};

// Workspace carving ----------------------------------------------------------
using kc_host::Plan;
using kc_host::align256;

size_t ws_size(const kc_graph *g, const Plan &p) { return kc_host::ws_bytes(g->n, p); }

struct Carved {
    WaveView wv;       // Wilson-wave view (B = BW), traversal fields point at sub-wave buffers
    int64_t *sids;
    int32_t *rs_q, *rs_pos;  // lane-to-warp hand-off of the hybrid walker
    unsigned int *done;
};

Carved carve(kc_graph *g, const Plan &p) {
    const size_t n = (size_t)g->n;
    char *base = (char *)g->d_ws;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        char *q = base + off;
        off += align256(bytes);
        return (void *)q;
    };
    Carved c;
    WaveView &w = c.wv;
    w.n = g->n;
    w.B = p.BW;
    w.word = (uint64_t *)take(sizeof(uint64_t) * n * p.BW);
    w.ord = (int32_t *)take(sizeof(int32_t) * n * p.BW);
    w.steps = (int64_t *)take(sizeof(int64_t) * p.BW);
    w.f = (int64_t *)take(sizeof(int64_t) * p.BW);
    c.sids = (int64_t *)take(sizeof(int64_t) * p.BW);
    c.rs_q = (int32_t *)take(sizeof(int32_t) * p.BW);
    c.rs_pos = (int32_t *)take(sizeof(int32_t) * p.BW);
    c.done = (unsigned int *)take(256);
    w.size = (int32_t *)take(sizeof(int32_t) * n * p.BT);
    w.vol = (int64_t *)take(sizeof(int64_t) * n * p.BT);
    w.din = (int32_t *)take(sizeof(int32_t) * n * p.BT);
    w.aux = (p.bit || p.canon) ? (int32_t *)take(sizeof(int32_t) * n * p.BT) : nullptr;
    w.bit = nullptr;
    w.stack = nullptr;
    w.stack_cap = p.stack_cap;
    if (p.bit) {
        w.bit = (int64_t *)take(sizeof(int64_t) * (n + 1) * p.BT);
        w.stack = g->d_stack;  // separate allocation, grown to BT x stack_cap entries
    }
    w.err = g->d_err;
    w.maxdepth = (int32_t *)(g->d_err + 1);
    return c;
}

// Workspaces come from the stream-ordered allocator on the handle's stream, so
// growing or releasing one never synchronises the device (handles on other
// streams keep running).
void ensure_ws(kc_graph *g, const Plan &p) {
    const size_t need = ws_size(g, p);
    if (need <= g->ws_bytes) return;
    if (g->d_ws) KC_CK(g, cudaFreeAsync(g->d_ws, g->stream));
    g->d_ws = nullptr;
    g->ws_bytes = 0;
    // 1% slack: plans for nearly equal tree counts fill the budget slightly
    // differently, and should not reallocate
    const size_t cap = need + need / 100;
    KC_CK(g, cudaMallocAsync(&g->d_ws, cap, g->stream));
    g->ws_bytes = cap;
}

void release_ws(kc_graph *g) {
    if (g->d_ws) KC_CK(g, cudaFreeAsync(g->d_ws, g->stream));
    if (g->d_stack) KC_CK(g, cudaFreeAsync(g->d_stack, g->stream));
    g->d_ws = nullptr;
    g->d_stack = nullptr;
    g->ws_bytes = 0;
    g->stack_bytes = 0;
}

// Pool growth (device arrays of per-tree values, optional parent arrays)
template <class T>
void grow(kc_graph *g, T *&p, int64_t old_count, int64_t new_cap, size_t per = 1) {
    T *q = nullptr;
    dalloc(g, &q, (size_t)new_cap * per);
    if (p && old_count > 0)
        KC_CK(g, cudaMemcpyAsync(q, p, sizeof(T) * (size_t)old_count * per,
                                 cudaMemcpyDeviceToDevice, g->stream));
    KC_CK(g, cudaStreamSynchronize(g->stream));
    dfree(p);
    p = q;
}

void ensure_pool(kc_graph *g, int64_t need) {
    if (need <= g->pool_cap) return;
    int64_t cap = std::max<int64_t>(need, std::max<int64_t>(1024, g->pool_cap * 2));
    if (g->cfg.keep_trees) cap = need;  // parent arrays are large: grow exactly
    grow(g, g->d_f, g->pool, cap);
    grow(g, g->d_w, g->pool, cap);
    grow(g, g->d_steps, g->pool, cap);
    grow(g, g->d_sid, g->pool, cap);
    if (g->cfg.keep_trees) grow(g, g->d_parents, g->pool, cap, (size_t)g->n);
    g->pool_cap = cap;
    g->h_modified.resize((size_t)cap, 0);
}

// Wave sizes within the workspace budget (kc_host_plan.h): the handle's cap,
// or a share of the device's free memory (counting the workspace it holds).
Plan plan_for(kc_graph *g, int64_t ntrees, bool canon = true, double walker_share = 0.7) {
    size_t free_b = 0, total_b = 0;
    KC_CK(g, cudaMemGetInfo(&free_b, &total_b));
    const double frac = g->cfg.mem_fraction > 0 ? g->cfg.mem_fraction : 0.8;
    const double budget = g->ws_limit > 0 ? (double)g->ws_limit
                                          : (double)(free_b + g->ws_bytes) * frac;
    return kc_host::plan_waves(g->n, ntrees, g->ttf_variant == KC_TTF_BIT, canon, budget,
                               g->cfg.max_trees_in_flight, walker_share);
}

// DFS stack of the BIT variant: one entry per stacked ancestor, so the
// deepest tree's depth + 2 entries per tree suffice.
void ensure_stack(kc_graph *g, Plan &p, uint32_t maxdepth, cudaStream_t st = nullptr) {
    if (!st) st = g->stream;
    const int64_t need_cap = (int64_t)maxdepth + 2;
    const size_t need = sizeof(int32_t) * 4 * (size_t)need_cap * (size_t)p.BT;
    if (need > g->stack_bytes) {
        if (g->d_stack) KC_CK(g, cudaFreeAsync(g->d_stack, st));
        g->d_stack = nullptr;
        g->stack_bytes = 0;
        KC_CK(g, cudaMallocAsync((void **)&g->d_stack, need, st));
        g->stack_bytes = need;
    }
    p.stack_cap = need_cap;
}

// Segmented BIT evaluation of f (k_ttf_bit_seg) -------------------------------

using kc_host::SegRegion;

int seg_limit(const kc_graph *g, int64_t b, bool walk_over) {
    return kc_host::seg_limit(g->cfg.ttf_segments, b, walk_over, g->num_sms);
}

// Segment tables for a wave of B trees: staging and device copies of
// B * max(16, cfg.ttf_segments) entries, taken from the start.
void reset_segtab(kc_graph *g, int64_t B) {
    const int64_t cap = B * std::max(16, g->cfg.ttf_segments);
    g->seg_used = 0;
    if (cap <= g->segtab_cap) return;
    // both streams are idle between waves: nothing reads the old tables
    KC_CK(g, cudaStreamSynchronize(g->stream));
    if (g->stream2) KC_CK(g, cudaStreamSynchronize(g->stream2));
    hfree(g->h_segtab);
    g->h_segtab = nullptr;
    dfree(g->d_segtab);
    g->d_segtab = nullptr;
    g->segtab_cap = 0;
    KC_CK(g, cudaMallocHost((void **)&g->h_segtab, sizeof(TtfSeg) * (size_t)cap));
    dalloc(g, &g->d_segtab, (size_t)cap);
    g->segtab_cap = cap;
}

// f of the b = sv.B trees of a sub-wave from k preorder segments per tree,
// k the largest value <= kmax for which b k Fenwick arrays (n int64, 8-byte
// aligned) and then b k stacks (stack_cap int4, 16-byte aligned) fit in
// `regions`; with grow (cfg.ttf_segments >= 2) the handle buffer d_segx holds
// kmax when they do not.  Segment j of a tree covers positions
// [j n / k, (j + 1) n / k).  Uploads the table and launches the segmented
// kernels on s; the caller has zeroed the trees' f.  Returns k, or 0 when fewer
// than two segments fit (the caller then runs the one-warp-per-tree kernel).
int ttf_bit_segmented(kc_graph *g, const GraphView &gv, const WaveView &sv, int kmax,
                      std::vector<SegRegion> regions, bool grow, cudaStream_t s) {
    const int64_t b = sv.B, n = g->n;
    if (kmax < 2 || b <= 0) return 0;
    const size_t bit_bytes = sizeof(int64_t) * (size_t)n;
    const size_t stk_bytes = sizeof(int4) * (size_t)sv.stack_cap;
    std::vector<uintptr_t> bits, stks;
    int k = kc_host::fit_segments(regions, b, kmax, bit_bytes, stk_bytes, bits, stks);
    if (k < kmax && grow) {
        const size_t want = (size_t)(b * kmax) * (bit_bytes + stk_bytes) + 64;
        if (want > g->segx_bytes) {
            if (g->d_segx) KC_CK(g, cudaFreeAsync(g->d_segx, s));
            g->d_segx = nullptr;
            g->segx_bytes = 0;
            KC_CK(g, cudaMallocAsync((void **)&g->d_segx, want, s));
            g->segx_bytes = want;
        }
        regions.assign(1, SegRegion{(uintptr_t)g->d_segx, g->segx_bytes});
        k = kmax;
        if (!kc_host::carve_segments(regions, (size_t)(b * k), bit_bytes, stk_bytes, bits,
                                     stks)) {
            g->last_error = "segmented BIT evaluation: buffer sizing";
            throw Fail{KC_ERR_CUDA};
        }
    }
    if (k < 2) return 0;
    if (g->seg_used + b * k > g->segtab_cap) {
        g->last_error = "segmented BIT evaluation: segment table overflow";
        throw Fail{KC_ERR_CUDA};
    }
    TtfSeg *h = g->h_segtab + g->seg_used;
    int64_t nseg = 0;
    for (int64_t t = 0; t < b; ++t)
        for (int j = 0; j < k; ++j) {
            const int64_t lo = j * n / k, hi = (j + 1) * n / k;
            if (lo == hi) continue;
            const size_t q = (size_t)(t * k + j);
            h[nseg++] = TtfSeg{(int64_t *)bits[q], (int4 *)stks[q], (int32_t)t, (int32_t)lo,
                               (int32_t)hi, 0};
        }
    TtfSeg *d = g->d_segtab + g->seg_used;
    g->seg_used += nseg;
    KC_CK(g, cudaMemcpyAsync(d, h, sizeof(TtfSeg) * (size_t)nseg, cudaMemcpyHostToDevice, s));
    KC_CK(g, launch_ttf_bit_seg(gv, sv, d, nseg, s));
    return k;
}

// Regions every BIT evaluation of a carved wave may reuse: the sub-wave
// Fenwick arrays (BT trees) and the stack buffer.  Only one chunk is evaluated
// at a time (one stream), so the next chunk finds them free again.
std::vector<SegRegion> subwave_regions(const kc_graph *g, const Plan &p, const WaveView &w) {
    std::vector<SegRegion> r;
    if (w.bit) r.push_back({(uintptr_t)w.bit, sizeof(int64_t) * (size_t)(g->n + 1) * (size_t)p.BT});
    if (g->d_stack) r.push_back({(uintptr_t)g->d_stack, g->stack_bytes});
    return r;
}

// BIT evaluation of a chunk: segmented when seg_limit allows and memory holds
// two or more segments a tree, else one warp per tree.  `walk_over`: the wave's
// walk has ended (its rejected trees' arrays, listed in `spare`, are free).
// Returns the kernels launched.
int eval_ttf_bit(kc_graph *g, const GraphView &gv, const Plan &p, const WaveView &sv,
                 bool walk_over, const std::vector<SegRegion> &spare, cudaStream_t s) {
    const int kmax = seg_limit(g, sv.B, walk_over);
    if (kmax >= 2) {
        std::vector<SegRegion> regs = subwave_regions(g, p, sv);
        if (walk_over) regs.insert(regs.end(), spare.begin(), spare.end());
        if (!sv.tmap)  // the segments add into f
            KC_CK(g, cudaMemsetAsync(sv.f, 0, sizeof(int64_t) * (size_t)sv.B, s));
        if (ttf_bit_segmented(g, gv, sv, kmax, std::move(regs), g->cfg.ttf_segments >= 2, s))
            return 2;
    }
    KC_CK(g, launch_ttf_bit(gv, sv, s));
    return 1;
}

// Cap on Wilson departures (per tree for the one-walker kernel, per walker for
// the 32-walker kernel): the configured value, or max(2^22, 1024 n) (about 60
// times the mean step count of a road-shaped graph, far above that of
// low-diameter graphs).
int64_t step_cap_of(const kc_graph *g) {
    if (g->cfg.step_cap > 0) return g->cfg.step_cap;
    return std::max<int64_t>((int64_t)1 << 22, 1024 * g->n);
}

// Traversal for f only: leaf-to-root atomics on large graphs with shallow trees
// (low eccentricity), the chunked warp-per-tree pass otherwise.
int fast_traversal(const kc_graph *g) {
    if (g->trav_mode >= 0) return g->trav_mode;
    return (g->ttf_variant == KC_TTF_SCAN && g->n >= (1 << 16)) ? kTravLeafUp : kTravChunked;
}

// Wilson's algorithm for the B trees of `w` (words and order already
// initialised, w.pos0 vertices placed) with the handle's walker.
void run_wilson(kc_graph *g, const GraphView &gv, const WaveView &w, const Carved &c) {
    const int64_t cap = step_cap_of(g);
    if (g->walker == KC_WALK_LANE) {
        KC_CK(g, launch_wilson(gv, w, g->seed, c.sids, cap, g->stream));
    } else if (g->walker == KC_WALK_WARP) {
        KC_CK(g, launch_wilson_warp(gv, w, g->seed, c.sids, g->d_sorder, cap, g->stream));
    } else {
        // lane walkers take the first starts of the hashed order (the long
        // early walks, where concurrent walkers would mostly wait on each
        // other); whatever is left, and lanes still running once most of the
        // wave has finished, continue with 32 walkers per tree
        const int pm = g->cfg.hybrid_prefix_permille > 0 ? g->cfg.hybrid_prefix_permille : 1000;
        const int tm = g->cfg.hybrid_tail_permille > 0 ? g->cfg.hybrid_tail_permille : 900;
        const int64_t q_stop = pm >= 1000 ? g->n : (g->n * pm) / 1000;
        const int64_t stop_at = tm >= 1000 ? 0 : std::max<int64_t>(1, (w.B * tm + 999) / 1000);
        KC_CK(g, cudaMemsetAsync(c.done, 0, sizeof(unsigned int), g->stream));
        KC_CK(g, launch_wilson(gv, w, g->seed, c.sids, cap, g->stream, g->d_sorder, c.rs_q,
                               c.rs_pos, c.done, q_stop, stop_at));
        KC_CK(g, launch_wilson_warp(gv, w, g->seed, c.sids, g->d_sorder, cap, g->stream, c.rs_q,
                                    c.rs_pos));
    }
}

int wilson_launches(const kc_graph *g) { return g->walker == KC_WALK_HYBRID ? 2 : 1; }

// One full sampling pass over sample ids [sid0, sid0 + B): walk, traverse,
// evaluate f.  Leaves per-tree results in the carved workspace.
// Completion flags (host-mapped), tree-map staging and the second stream of
// pipelined waves, sized for B trees.
void ensure_pipeline(kc_graph *g, int64_t B) {
    if (!g->stream2) KC_CK(g, cudaStreamCreateWithFlags(&g->stream2, cudaStreamNonBlocking));
    if (B <= g->done_cap) return;
    hfree(g->h_done);
    hfree(g->h_map);
    hfree(g->h_segtab);
    dfree(g->d_segtab);
    dfree(g->d_segx);
    dfree(g->d_map);
    g->h_done = g->h_map = g->d_done = nullptr;
    g->done_cap = 0;
    KC_CK(g, cudaHostAlloc((void **)&g->h_done, sizeof(int32_t) * (size_t)B, cudaHostAllocMapped));
    KC_CK(g, cudaHostGetDevicePointer((void **)&g->d_done, g->h_done, 0));
    KC_CK(g, cudaMallocHost((void **)&g->h_map, sizeof(int32_t) * (size_t)B));
    dalloc(g, &g->d_map, (size_t)B);
    g->done_cap = B;
}

// A wave whose traversal and TTF start on a second stream while the walk is
// still running: the 32-walker kernel flags every finished tree in host-mapped
// memory, the host gathers finished trees into chunks of up to BT (a tree map
// per chunk) and launches their sub-wave kernels; only the chunk holding the
// slowest trees waits for the end of the walk.
// With reject, the walk abandons trees past cfg.reject_steps departures; they
// flag -1 and are left out of the chunks (their f stays 0, their steps -1).
void run_wave_pipelined(kc_graph *g, Plan &p, int64_t B, int64_t sid0, bool reject = false) {
    ensure_pipeline(g, B);
    GraphView gv = view_of(g);
    Carved c = carve(g, p);
    WaveView w = c.wv;
    w.B = B;
    cudaStream_t s1 = g->stream, s2 = g->stream2;
    std::vector<cudaEvent_t> evs;
    auto event = [&]() {
        cudaEvent_t e = nullptr;
        KC_CK(g, cudaEventCreate(&e));
        evs.push_back(e);
        return e;
    };
    struct EvGuard {
        std::vector<cudaEvent_t> &v;
        ~EvGuard() {
            for (cudaEvent_t e : v) cudaEventDestroy(e);
        }
    } guard{evs};
    volatile int32_t *hd = g->h_done;
    for (int64_t t = 0; t < B; ++t) hd[t] = 0;
    reset_segtab(g, B);
    std::vector<SegRegion> spare;  // walk arrays of rejected trees (free once the walk ended)
    KC_CK(g, cudaMemsetAsync(g->d_err, 0, 2 * sizeof(uint32_t), s1));
    KC_CK(g, cudaMemsetAsync(w.f, 0, sizeof(int64_t) * (size_t)B, s1));
    KC_CK(g, launch_iota(c.sids, sid0, B, s1));
    {
        Phase ph(g, g->t_init);
        KC_CK(g, launch_wave_init(gv, w, s1));
        ph.done(1);
    }
    cudaEvent_t ev_ready = event(), ev_w0 = event(), ev_w1 = event();
    KC_CK(g, cudaEventRecord(ev_ready, s1));
    KC_CK(g, cudaStreamWaitEvent(s2, ev_ready, 0));
    KC_CK(g, cudaEventRecord(ev_w0, s1));
    if (g->walker == KC_WALK_LANE) {
        if (reject)
            KC_CK(g, launch_wilson_reject(gv, w, g->seed, c.sids, nullptr, g->cfg.reject_steps,
                                          s1, g->d_done));
        else
            KC_CK(g, launch_wilson(gv, w, g->seed, c.sids, step_cap_of(g), s1, nullptr, nullptr,
                                   nullptr, nullptr, 0, 0, g->d_done));
    } else if (reject) {
        KC_CK(g, launch_wilson_warp_reject(gv, w, g->seed, c.sids, g->d_sorder,
                                           g->cfg.reject_steps, s1, g->d_done));
    } else {
        KC_CK(g, launch_wilson_warp(gv, w, g->seed, c.sids, g->d_sorder, step_cap_of(g), s1,
                                    nullptr, nullptr, g->d_done));
    }
    KC_CK(g, cudaEventRecord(ev_w1, s1));
    const int64_t chunk_min = std::max<int64_t>(1, std::min<int64_t>(p.BT, (B + 1) / 2));
    std::vector<int32_t> unseen((size_t)B), ready;
    for (int64_t t = 0; t < B; ++t) unseen[(size_t)t] = (int32_t)t;
    std::vector<std::array<cudaEvent_t, 3>> chunk_ev;
    int64_t processed = 0, skipped = 0;  // trees put into chunks / rejected
    bool wdone = false;
    while (processed + skipped < B) {
        if (!wdone) {
            const cudaError_t q = cudaEventQuery(ev_w1);
            if (q == cudaSuccess) wdone = true;
            else if (q != cudaErrorNotReady) KC_CK(g, q);
        }
        size_t keep = 0;
        for (size_t i = 0; i < unseen.size(); ++i) {
            const int32_t t = unseen[i];
            const int32_t flag = hd[t];
            if (flag > 0) {
                ready.push_back(t);
            } else if (flag < 0) {
                ++skipped;
                spare.push_back({(uintptr_t)(w.word + (int64_t)t * g->n), sizeof(uint64_t) * (size_t)g->n});
                spare.push_back({(uintptr_t)(w.ord + (int64_t)t * g->n), sizeof(int32_t) * (size_t)g->n});
            } else {
                unseen[keep++] = t;
            }
        }
        unseen.resize(keep);
        if ((int64_t)ready.size() >= (wdone ? 1 : chunk_min)) {
            const int64_t b = std::min<int64_t>(p.BT, (int64_t)ready.size());
            int32_t md = 0;
            for (int64_t k = 0; k < b; ++k) {
                const int32_t t = ready[(size_t)k];
                g->h_map[processed + k] = t;
                md = std::max(md, hd[t] - 1);
            }
            ready.erase(ready.begin(), ready.begin() + b);
            KC_CK(g, cudaMemcpyAsync(g->d_map + processed, g->h_map + processed,
                                     sizeof(int32_t) * (size_t)b, cudaMemcpyHostToDevice, s2));
            if (p.bit) {
                ensure_stack(g, p, (uint32_t)md, s2);
                c = carve(g, p);
            }
            WaveView sv = c.wv;
            sv.B = b;
            sv.tmap = g->d_map + processed;
            std::array<cudaEvent_t, 3> e3 = {event(), event(), event()};
            KC_CK(g, cudaEventRecord(e3[0], s2));
            int nl = 0;
            KC_CK(g, launch_traverse(gv, sv, p.bit, s2, &nl, fast_traversal(g)));
            g->t_traverse.launches += nl;
            KC_CK(g, cudaEventRecord(e3[1], s2));
            if (p.bit) g->t_ttf.launches += eval_ttf_bit(g, gv, p, sv, wdone, spare, s2);
            else {
                KC_CK(g, launch_ttf_scan(gv, sv, s2));
                g->t_ttf.launches += 1;
            }
            KC_CK(g, cudaEventRecord(e3[2], s2));
            chunk_ev.push_back(e3);
            processed += b;
            continue;
        }
        if (wdone && unseen.empty() && ready.empty()) break;
        if (wdone && !unseen.empty()) {
            // the walk is over: every flag is visible now
            bool any = false;
            for (int32_t t : unseen) any = any || hd[t] != 0;
            if (!any) {
                g->last_error = "a walker finished without flagging its tree";
                throw Fail{KC_ERR_CUDA};
            }
            continue;
        }
        std::this_thread::sleep_for(std::chrono::microseconds(100));
    }
    cudaEvent_t ev_join = event();
    KC_CK(g, cudaEventRecord(ev_join, s2));
    KC_CK(g, cudaStreamWaitEvent(s1, ev_join, 0));
    KC_CK(g, cudaStreamSynchronize(s1));
    float ms = 0.f;
    KC_CK(g, cudaEventElapsedTime(&ms, ev_w0, ev_w1));
    g->t_wilson.ms += ms;
    g->t_wilson.launches += 1;
    for (auto &e3 : chunk_ev) {
        KC_CK(g, cudaEventElapsedTime(&ms, e3[0], e3[1]));
        g->t_traverse.ms += ms;
        KC_CK(g, cudaEventElapsedTime(&ms, e3[1], e3[2]));
        g->t_ttf.ms += ms;
    }
    uint32_t hdr[2] = {0, 0};
    KC_CK(g, copy_sync(g, hdr, g->d_err, sizeof(hdr), cudaMemcpyDeviceToHost));
    if (hdr[0] & kErrStepLimit) {
        g->last_error = "Wilson walk exceeded the step cap";
        throw Fail{KC_ERR_STEP_LIMIT};
    }
    if (hdr[0] & (kErrBadTree | kErrIterLimit)) {
        g->last_error = "inconsistent tree state, walker iteration cap or traversal stack overflow";
        throw Fail{KC_ERR_CUDA};
    }
}

void run_wave(kc_graph *g, Plan &p, int64_t B, int64_t sid0, bool canonical = false) {
    // pipelining pays when traversal and TTF take long enough to hide: several
    // sub-waves, or large graphs; short waves of small graphs run straight
    if (!canonical && !g->tuning && (g->walker == KC_WALK_WARP || g->walker == KC_WALK_LANE) &&
        B > 1 &&
        (B > p.BT || g->n >= (1 << 16))) {
        try {
            run_wave_pipelined(g, p, B, sid0);
        } catch (Fail &) {
            // let both streams drain before the workspace is reused
            cudaStreamSynchronize(g->stream);
            if (g->stream2) cudaStreamSynchronize(g->stream2);
            throw;
        }
        return;
    }
    GraphView gv = view_of(g);
    Carved c = carve(g, p);
    WaveView w = c.wv;
    w.B = B;
    KC_CK(g, cudaMemsetAsync(g->d_err, 0, 2 * sizeof(uint32_t), g->stream));
    KC_CK(g, launch_iota(c.sids, sid0, B, g->stream));
    reset_segtab(g, B);
    {
        Phase ph(g, g->t_init);
        KC_CK(g, launch_wave_init(gv, w, g->stream));
        ph.done(1);
    }
    {
        Phase ph(g, g->t_wilson);
        run_wilson(g, gv, w, c);
        ph.done(wilson_launches(g));
    }
    uint32_t hdr[2] = {0, 0};
    KC_CK(g, copy_sync(g, hdr, g->d_err, sizeof(hdr), cudaMemcpyDeviceToHost));
    if (hdr[0] & kErrStepLimit) {
        g->last_error = "Wilson walk exceeded the step cap";
        throw Fail{KC_ERR_STEP_LIMIT};
    }
    if (hdr[0] & (kErrBadTree | kErrIterLimit)) {
        g->last_error = "Wilson walkers reached an inconsistent state or the iteration cap";
        throw Fail{KC_ERR_CUDA};
    }
    if (p.bit) {
        ensure_stack(g, p, hdr[1]);
        c = carve(g, p);
        w = c.wv;
        w.B = B;
    }
    for (int64_t sub = 0; sub < B; sub += p.BT) {
        const int64_t b = std::min<int64_t>(p.BT, B - sub);
        WaveView s = w;
        s.B = b;
        s.word = w.word + sub * g->n;
        s.ord = w.ord + sub * g->n;
        s.steps = w.steps + sub;
        s.f = w.f + sub;
        {
            Phase ph(g, g->t_traverse);
            int nl = 0;
            KC_CK(g, launch_traverse(gv, s, p.bit, g->stream, &nl,
                                     canonical ? kTravCanonical : fast_traversal(g)));
            ph.done(nl);
        }
        {
            Phase ph(g, g->t_ttf);
            int nl = 1;
            if (p.bit) nl = eval_ttf_bit(g, gv, p, s, true, {}, g->stream);
            else KC_CK(g, launch_ttf_scan(gv, s, g->stream));
            ph.done(nl);
        }
    }
    KC_CK(g, copy_sync(g, hdr, g->d_err, sizeof(hdr), cudaMemcpyDeviceToHost));
    if (hdr[0] & kErrBadTree) {
        g->last_error = "inconsistent tree state or traversal stack overflow";
        throw Fail{KC_ERR_CUDA};
    }
}



// BFS levels from src into `level` (one launch per level)
void bfs_levels_dev(kc_graph *g, int32_t src, int32_t *level, int &launches) {
    GraphView gv = view_of(g);
    KC_CK(g, launch_bfs_init(g->n, src, level, g->stream));
    ++launches;
    int32_t *d_changed = (int32_t *)g->d_scratch;
    for (int32_t lev = 0;; ++lev) {
        KC_CK(g, cudaMemsetAsync(d_changed, 0, sizeof(int32_t), g->stream));
        KC_CK(g, launch_bfs_level(gv, lev, level, d_changed, g->stream));
        ++launches;
        int32_t changed = 0;
        KC_CK(g, cudaMemcpyAsync(&changed, d_changed, sizeof(changed), cudaMemcpyDeviceToHost,
                                 g->stream));
        KC_CK(g, cudaStreamSynchronize(g->stream));
        if (!changed) break;
        if (lev > g->n) throw Fail{KC_ERR_CUDA};
    }
}

unsigned long long argmax_dev(kc_graph *g, const int32_t *la, const int32_t *lb, int mode,
                              int &launches) {
    unsigned long long *d = (unsigned long long *)g->d_scratch + 8;
    KC_CK(g, cudaMemsetAsync(d, 0, sizeof(unsigned long long), g->stream));
    KC_CK(g, launch_argmax_score(g->n, la, lb, mode, d, g->stream));
    ++launches;
    unsigned long long h = 0;
    KC_CK(g, cudaMemcpyAsync(&h, d, sizeof(h), cudaMemcpyDeviceToHost, g->stream));
    KC_CK(g, cudaStreamSynchronize(g->stream));
    return h;
}

// Highest-degree vertex, ties broken towards the centre (the paper fixes no
// tie-break; Exp-III prefers the root that shortens the walks): with r0 the
// smallest-id highest-degree vertex, a the vertex farthest from r0, b the
// vertex farthest from a and c the vertex maximising min(dist(a,.), dist(b,.)),
// the root minimises max(dist(a,.), dist(b,.), dist(c,.)) over the
// highest-degree vertices, smallest id among equals.  Unique maximum: r0.
int32_t central_root(kc_graph *g, int32_t r0, int &launches) {
    int32_t dmax = 0;
    KC_CK(g, copy_sync(g, &dmax, g->d_deg + r0, sizeof(int32_t), cudaMemcpyDeviceToHost));
    int32_t *d_ties = (int32_t *)g->d_scratch + 32;
    unsigned long long *d_best = (unsigned long long *)g->d_scratch + 24;
    KC_CK(g, cudaMemsetAsync(d_ties, 0, sizeof(int32_t), g->stream));
    KC_CK(g, launch_central_pick(g->n, g->d_deg, dmax, nullptr, nullptr, nullptr, d_best, d_ties,
                                 g->stream));
    ++launches;
    int32_t ties = 0;
    KC_CK(g, cudaMemcpyAsync(&ties, d_ties, sizeof(int32_t), cudaMemcpyDeviceToHost, g->stream));
    KC_CK(g, cudaStreamSynchronize(g->stream));
    if (ties <= 1) return r0;
    int32_t *lv = nullptr;
    dalloc(g, &lv, (size_t)(3 * g->n));
    int32_t *la = lv, *lb = lv + g->n, *lc = lv + 2 * g->n;
    try {
        bfs_levels_dev(g, r0, la, launches);
        const int32_t a = (int32_t)(0xFFFFFFFFull - (argmax_dev(g, la, la, 0, launches) & 0xFFFFFFFFull));
        bfs_levels_dev(g, a, la, launches);
        const int32_t b = (int32_t)(0xFFFFFFFFull - (argmax_dev(g, la, la, 0, launches) & 0xFFFFFFFFull));
        bfs_levels_dev(g, b, lb, launches);
        const int32_t c = (int32_t)(0xFFFFFFFFull - (argmax_dev(g, la, lb, 1, launches) & 0xFFFFFFFFull));
        bfs_levels_dev(g, c, lc, launches);
        KC_CK(g, cudaMemsetAsync(d_best, 0xFF, sizeof(unsigned long long), g->stream));
        KC_CK(g, launch_central_pick(g->n, g->d_deg, dmax, la, lb, lc, d_best, d_ties, g->stream));
        ++launches;
        unsigned long long best = 0;
        KC_CK(g, cudaMemcpyAsync(&best, d_best, sizeof(best), cudaMemcpyDeviceToHost, g->stream));
        KC_CK(g, cudaStreamSynchronize(g->stream));
        dfree(lv);
        return (int32_t)(best & 0xFFFFFFFFull);
    } catch (Fail &) {
        dfree(lv);
        throw;
    }
}

// tau0 = BFS tree from g->root over the current device graph (parent = the
// smallest-id neighbour one level closer), level-synchronous, one launch per
// level; sets g->ecc.  Throws KC_ERR_DISCONNECTED if a vertex is unreached.
void build_tau0_bfs(kc_graph *g, int &launches) {
    GraphView gv = view_of(g);
    const int64_t n = g->n;
    KC_CK(g, launch_bfs_init(n, g->root, g->d_level0, g->stream));
    ++launches;
    int32_t *d_changed = (int32_t *)g->d_scratch;
    int32_t lev = 0;
    for (;; ++lev) {
        KC_CK(g, cudaMemsetAsync(d_changed, 0, sizeof(int32_t), g->stream));
        KC_CK(g, launch_bfs_level(gv, lev, g->d_level0, d_changed, g->stream));
        ++launches;
        int32_t changed = 0;
        KC_CK(g, cudaMemcpyAsync(&changed, d_changed, sizeof(changed), cudaMemcpyDeviceToHost,
                                 g->stream));
        KC_CK(g, cudaStreamSynchronize(g->stream));
        if (!changed) break;
        if (lev > n) throw Fail{KC_ERR_CUDA};
    }
    g->ecc = lev;
    gv.ecc = lev;
    int32_t *d_unreached = (int32_t *)g->d_scratch;
    KC_CK(g, cudaMemsetAsync(d_unreached, 0, sizeof(int32_t), g->stream));
    KC_CK(g, launch_bfs_parent(gv, g->d_level0, g->d_p0, d_unreached, g->stream));
    ++launches;
    int32_t unreached = 0;
    KC_CK(g, cudaMemcpyAsync(&unreached, d_unreached, sizeof(int32_t), cudaMemcpyDeviceToHost,
                             g->stream));
    KC_CK(g, cudaStreamSynchronize(g->stream));
    if (unreached) throw Fail{KC_ERR_DISCONNECTED};
}

// Exp-II's depth-first path tree: one device thread, explicit stack.
void build_tau0_dfs(kc_graph *g, int &launches) {
    GraphView gv = view_of(g);
    const int64_t n = g->n;
    int32_t *sv = nullptr;
    int64_t *se = nullptr;
    KC_CK(g, cudaMallocAsync((void **)&sv, sizeof(int32_t) * (size_t)n, g->stream));
    KC_CK(g, cudaMallocAsync((void **)&se, sizeof(int64_t) * (size_t)n, g->stream));
    int32_t *d_cnt = (int32_t *)g->d_scratch;  // [0] deepest, [1] unreached
    KC_CK(g, cudaMemsetAsync(d_cnt, 0, 2 * sizeof(int32_t), g->stream));
    KC_CK(g, launch_dfs_tree(gv, g->root, g->d_p0, g->d_level0, sv, se, d_cnt, d_cnt + 1,
                             g->stream));
    launches += 3;
    KC_CK(g, cudaFreeAsync(sv, g->stream));
    KC_CK(g, cudaFreeAsync(se, g->stream));
    int32_t h[2] = {0, 0};
    KC_CK(g, copy_sync(g, h, d_cnt, sizeof(h), cudaMemcpyDeviceToHost));
    if (h[1]) throw Fail{KC_ERR_DISCONNECTED};
    g->ecc = h[0];
}

// Exp-II's Wilson path tree: the uniform tree of sample id 0 under tau0_seed,
// drawn by the 32-walker kernel; its parents and depths become p0 and level.
void build_tau0_wilson(kc_graph *g, int &launches) {
    GraphView gv = view_of(g);
    Plan p;
    p.BW = 1;
    p.BT = 1;
    ensure_ws(g, p);
    Carved c = carve(g, p);
    WaveView w = c.wv;
    w.B = 1;
    KC_CK(g, cudaMemsetAsync(g->d_err, 0, 2 * sizeof(uint32_t), g->stream));
    KC_CK(g, launch_iota(c.sids, 0, 1, g->stream));
    KC_CK(g, launch_wave_init(gv, w, g->stream));
    KC_CK(g, launch_wilson_warp(gv, w, g->cfg.tau0_seed, c.sids, g->d_sorder, step_cap_of(g),
                                g->stream));
    int32_t *d_cnt = (int32_t *)g->d_scratch;  // [0] deepest, [1] outside the tree
    KC_CK(g, cudaMemsetAsync(d_cnt, 0, 2 * sizeof(int32_t), g->stream));
    KC_CK(g, launch_tau0_from_words(g->n, w.word, g->d_p0, g->d_level0, d_cnt, d_cnt + 1,
                                    g->stream));
    launches += 4;
    uint32_t hdr[2] = {0, 0};
    KC_CK(g, copy_sync(g, hdr, g->d_err, sizeof(hdr), cudaMemcpyDeviceToHost));
    if (hdr[0] & kErrStepLimit) {
        g->last_error = "the Wilson path tree exceeded the step cap";
        throw Fail{KC_ERR_STEP_LIMIT};
    }
    if (hdr[0]) throw Fail{KC_ERR_CUDA};
    int32_t h[2] = {0, 0};
    KC_CK(g, copy_sync(g, h, d_cnt, sizeof(h), cudaMemcpyDeviceToHost));
    if (h[1]) throw Fail{KC_ERR_DISCONNECTED};
    g->ecc = h[0];
}

void build_tau0(kc_graph *g, int &launches) {
    if (g->cfg.tau0_kind == KC_TAU0_DFS) build_tau0_dfs(g, launches);
    else if (g->cfg.tau0_kind == KC_TAU0_WILSON) build_tau0_wilson(g, launches);
    else build_tau0_bfs(g, launches);
}

// DFN of tau0 with the same passes as the sampled trees (one tree).
void traverse_tau0(kc_graph *g, int &launches) {
    GraphView gv = view_of(g);
    const int64_t n = g->n;
    Plan p;
    p.BW = 1;
    p.BT = 1;
    ensure_ws(g, p);
    Carved c = carve(g, p);
    WaveView w = c.wv;
    w.B = 1;
    KC_CK(g, launch_tau0_words(n, g->d_p0, g->d_level0, w.word, g->stream));
    KC_CK(g, launch_level_order(n, g->ecc, g->d_level0, w.din, w.ord, g->stream));
    int nl = 0;
    KC_CK(g, launch_traverse(gv, w, false, g->stream, &nl));
    KC_CK(g, launch_out_from_size(n, w.din, w.size, g->d_out0, g->stream));
    KC_CK(g, cudaMemcpyAsync(g->d_in0, w.din, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice,
                             g->stream));
    launches += 4 + nl;
}

// ===========================================================================
// Sample maintenance (Algorithms 2 and 3)
// ===========================================================================
// |f| <= 4 m^2 ecc(r) (Theorem 5's proof) must stay below 2^62 for the int64 f
bool f_may_overflow(int64_t m, int32_t ecc) {
    const long double bound = 4.0L * (long double)m * (long double)m * (long double)ecc;
    return bound >= 4611686018427387904.0L;
}

// The whole batch against the evolving graph, before anything is applied.  The
// graph is connected before the batch and every accepted op keeps it so; a
// deletion then keeps it connected exactly when its endpoints stay connected.
// Insertions keep tau0 (and ecc) and grow m, so the overflow margin is checked
// for each; a deletion that rebuilds tau0 is checked when the new ecc is known.
kc_status validate_batch(kc_graph *g, const kc_edge_op *ops, int64_t n_ops) {
    kc_host::OverlayGraph og(g->h_row_off.data(), g->h_col.data(), g->n);
    int64_t m = g->m;
    for (int64_t i = 0; i < n_ops; ++i) {
        const kc_edge_op &o = ops[i];
        if (o.u < 0 || o.v < 0 || o.u >= g->n || o.v >= g->n || o.u == o.v ||
            (o.op != 0 && o.op != 1))
            return KC_ERR_INVALID_ARG;
        if (o.op == 0 && g->cfg.r_source == KC_R_GIVEN && !(o.r > 0.0 && o.r <= 1.0))
            return KC_ERR_INVALID_ARG;
        const bool present = og.has_edge(o.u, o.v);
        if (o.op == 0 && present) return KC_ERR_EDGE_EXISTS;
        if (o.op == 1 && !present) return KC_ERR_EDGE_MISSING;
        if (o.op == 0) {
            og.insert(o.u, o.v);
            if (f_may_overflow(++m, g->ecc)) return KC_ERR_OVERFLOW;
        } else {
            og.erase(o.u, o.v);
            if (!og.connected(o.u, o.v)) return KC_ERR_BRIDGE;
            --m;
        }
    }
    return KC_OK;
}

// Host wall time of one part of an update (every part ends synchronised).
struct UpdPart {
    double &acc;
    std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
    explicit UpdPart(double &a) : acc(a) {}
    ~UpdPart() {
        acc += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0)
                   .count();
    }
};

// One op on the device CSR (rows kept sorted), then the walk records and
// degrees of the changed graph; the host copy of the CSR is refreshed once per
// batch (sync_host_csr).  Nothing goes through the host per op but the check
// that the edit applied.
void edit_graph(kc_graph *g, int32_t u, int32_t v, bool insert) {
    const int64_t twom = 2 * g->m;
    const size_t need = (size_t)twom + 2;
    if (need > g->col_cap) {
        const size_t cap = need + need / 8 + 64;
        int32_t *q = nullptr;
        dalloc(g, &q, cap);
        KC_CK(g, cudaMemcpyAsync(q, g->d_col, sizeof(int32_t) * (size_t)twom,
                                 cudaMemcpyDeviceToDevice, g->stream));
        KC_CK(g, cudaStreamSynchronize(g->stream));
        dfree(g->d_col);
        g->d_col = q;
        g->col_cap = cap;
    }
    if (need > g->edit_cap) {
        dfree(g->d_edit);
        const size_t cap = std::max(need + need / 8 + 64, g->col_cap);
        dalloc(g, &g->d_edit, cap);
        g->edit_cap = cap;
    }
    int64_t *pos = (int64_t *)g->d_scratch + 64;  // 3 words past the reduction sums
    KC_CK(g, launch_csr_edit(g->n, twom, g->d_row_off, g->d_col, g->d_edit, pos, u, v, insert,
                             g->stream));
    int64_t hp[3] = {0, 0, 0};
    KC_CK(g, copy_sync(g, hp, pos, sizeof(hp), cudaMemcpyDeviceToHost));
    if (hp[2]) {
        g->last_error = "kc_update: the device graph does not match the validated batch";
        throw Fail{KC_ERR_CUDA};
    }
    g->m += insert ? 1 : -1;
    g->host_csr_stale = true;
    KC_CK(g, launch_build_records(view_of(g), g->d_rec, g->d_deg, g->stream));
    g->t_update.launches += 4;
}

// the host copy of the CSR (batch validation reads it) from the device
void sync_host_csr(kc_graph *g) {
    if (!g->host_csr_stale) return;
    const int64_t n = g->n;
    g->h_row_off.resize((size_t)n + 1);
    KC_CK(g, copy_sync(g, g->h_row_off.data(), g->d_row_off, sizeof(int64_t) * (size_t)(n + 1),
                       cudaMemcpyDeviceToHost));
    const int64_t twom = g->h_row_off[(size_t)n];
    g->h_col.resize((size_t)twom);
    KC_CK(g, copy_sync(g, g->h_col.data(), g->d_col, sizeof(int32_t) * (size_t)twom,
                       cudaMemcpyDeviceToHost));
    g->host_csr_stale = false;
}

struct UpdBuf {
    int64_t *slots;   // [P]
    double *factor;   // [P]
    int64_t *sel;     // [P]
    uint8_t *flags;   // [P]
    uint8_t *taken;   // [P]
    double *sums;     // [4]
};

UpdBuf upd_buf(kc_graph *g) {
    const size_t P = (size_t)std::max<int64_t>(g->pool, 1);
    const size_t need = align256(8 * P) * 3 + align256(P) * 2 + 256;
    if (need > g->ub_bytes) {
        if (g->d_ub) cudaFree(g->d_ub);
        g->d_ub = nullptr;
        g->ub_bytes = 0;
        KC_CK(g, cudaMalloc(&g->d_ub, need));
        g->ub_bytes = need;
    }
    char *b = (char *)g->d_ub;
    UpdBuf u;
    u.slots = (int64_t *)b;
    b += align256(8 * P);
    u.factor = (double *)b;
    b += align256(8 * P);
    u.sel = (int64_t *)b;
    b += align256(8 * P);
    u.flags = (uint8_t *)b;
    b += align256(P);
    u.taken = (uint8_t *)b;
    b += align256(P);
    u.sums = (double *)b;
    return u;
}

void check_err(kc_graph *g, const char *what) {
    uint32_t hdr[2] = {0, 0};
    KC_CK(g, copy_sync(g, hdr, g->d_err, sizeof(hdr), cudaMemcpyDeviceToHost));
    if (hdr[0] & kErrStepLimit) {
        g->last_error = std::string(what) + ": Wilson walk exceeded the step cap";
        throw Fail{KC_ERR_STEP_LIMIT};
    }
    if (hdr[0]) {
        g->last_error = std::string(what) + ": inconsistent tree state";
        throw Fail{KC_ERR_CUDA};
    }
}

// traversal and f(tau) of the retained trees at `slots`, on the current graph
void refresh_slots(kc_graph *g, const std::vector<int64_t> &slots) {
    if (slots.empty()) return;
    UpdPart tp(g->ms_upd_part[3]);
    GraphView gv = view_of(g);
    Plan p = plan_for(g, (int64_t)slots.size());
    ensure_ws(g, p);
    UpdBuf ub = upd_buf(g);
    for (size_t c0 = 0; c0 < slots.size(); c0 += (size_t)p.BT) {
        const int64_t b = std::min<int64_t>(p.BT, (int64_t)(slots.size() - c0));
        KC_CK(g, cudaMemcpyAsync(ub.slots, slots.data() + c0, sizeof(int64_t) * b,
                                 cudaMemcpyHostToDevice, g->stream));
        KC_CK(g, cudaMemsetAsync(g->d_err, 0, 2 * sizeof(uint32_t), g->stream));
        Carved c = carve(g, p);
        WaveView w = c.wv;
        w.B = b;
        KC_CK(g, launch_prepare_from_parents(g->n, b, g->root, g->d_parents, ub.slots, w,
                                             g->stream));
        uint32_t hdr[2] = {0, 0};
        KC_CK(g, cudaMemcpyAsync(hdr, g->d_err, sizeof(hdr), cudaMemcpyDeviceToHost, g->stream));
        KC_CK(g, cudaStreamSynchronize(g->stream));
        if (hdr[0]) check_err(g, "refresh");
        if (p.bit) {
            ensure_stack(g, p, hdr[1]);
            c = carve(g, p);
            w = c.wv;
            w.B = b;
        }
        int nl = 0;
        KC_CK(g, launch_traverse(gv, w, p.bit, g->stream, &nl, fast_traversal(g)));
        if (p.bit) KC_CK(g, launch_ttf_bit(gv, w, g->stream));
        else KC_CK(g, launch_ttf_scan(gv, w, g->stream));
        KC_CK(g, launch_scatter_results(ub.slots, b, w.f, nullptr, nullptr, g->d_f, g->d_steps,
                                        g->d_sid, g->stream));
        g->t_update.launches += nl + 6;
        check_err(g, "refresh");
    }
}

// replace the retained trees at `slots` by fresh trees with new sample ids
// (in slot order): uniform trees of the current graph, or, with cond, uniform
// trees conditioned on containing (u, v), re-rooted at r
void resample_slots(kc_graph *g, const std::vector<int64_t> &slots, bool cond, int32_t u,
                    int32_t v) {
    if (slots.empty()) return;
    GraphView gv = view_of(g);
    Plan p = plan_for(g, (int64_t)slots.size());
    ensure_ws(g, p);
    UpdBuf ub = upd_buf(g);
    const int64_t chunk = std::min(p.BW, p.BT);
    for (size_t c0 = 0; c0 < slots.size(); c0 += (size_t)chunk) {
        const int64_t b = std::min<int64_t>(chunk, (int64_t)(slots.size() - c0));
        KC_CK(g, cudaMemcpyAsync(ub.slots, slots.data() + c0, sizeof(int64_t) * b,
                                 cudaMemcpyHostToDevice, g->stream));
        KC_CK(g, cudaMemsetAsync(g->d_err, 0, 2 * sizeof(uint32_t), g->stream));
        Carved c = carve(g, p);
        WaveView w = c.wv;
        w.B = b;
        KC_CK(g, launch_iota(c.sids, g->next_sid, b, g->stream));
        if (cond) {
            KC_CK(g, launch_edge_pre_init(g->n, b, u, v, w.word, w.ord, g->stream));
            w.pos0 = 2;
        } else {
            KC_CK(g, launch_wave_init(gv, w, g->stream));
            w.pos0 = 1;
        }
        run_wilson(g, gv, w, c);
        KC_CK(g, launch_words_to_slots(g->n, b, w.word, ub.slots, g->d_parents, g->root,
                                       cond ? v : -1, g->d_err, g->stream));
        KC_CK(g, launch_scatter_results(ub.slots, b, nullptr, w.steps, c.sids, g->d_f,
                                        g->d_steps, g->d_sid, g->stream));
        check_err(g, "resample");
        g->next_sid += b;
        g->t_update.launches += 4 + wilson_launches(g);
        std::vector<int64_t> part(slots.begin() + c0, slots.begin() + c0 + b);
        for (int64_t x : part) g->h_modified[(size_t)x] = 1;
        refresh_slots(g, part);
    }
    g->trees_resampled += (int64_t)slots.size();
}

// ISM: link-cut (insert) or cut-link (delete) of the trees at `slots`, their
// weights multiplied by d_old / d_new, then their f recomputed
void transform_slots(kc_graph *g, const std::vector<int64_t> &slots, bool insert, int32_t u,
                     int32_t v) {
    if (slots.empty()) return;
    GraphView gv = view_of(g);
    Plan p = plan_for(g, (int64_t)slots.size());
    ensure_ws(g, p);
    UpdBuf ub = upd_buf(g);
    for (size_t c0 = 0; c0 < slots.size(); c0 += (size_t)p.BT) {
        const int64_t b = std::min<int64_t>(p.BT, (int64_t)(slots.size() - c0));
        KC_CK(g, cudaMemcpyAsync(ub.slots, slots.data() + c0, sizeof(int64_t) * b,
                                 cudaMemcpyHostToDevice, g->stream));
        KC_CK(g, cudaMemsetAsync(g->d_err, 0, 2 * sizeof(uint32_t), g->stream));
        Carved c = carve(g, p);
        WaveView w = c.wv;
        w.B = b;
        KC_CK(g, launch_prepare_from_parents(g->n, b, g->root, g->d_parents, ub.slots, w,
                                             g->stream));
        // link-cut reads the DFN only to test subtree membership, so any valid
        // DFN serves (the warp-per-tree pass); cut-link picks the k-th crossing
        // edge in the id-ordered preorder, which the canonical pass gives
        int nl = 0;
        KC_CK(g, launch_traverse(gv, w, true, g->stream, &nl,
                                 insert ? kTravChunked : kTravCanonical));
        KC_CK(g, launch_link_cut(g->d_row_off, g->d_col, w, ub.slots, g->d_parents, ub.factor,
                                 g->root, u, v, g->seed, (uint32_t)g->update_seq, insert,
                                 g->stream));
        KC_CK(g, launch_scale_slots(g->d_w, ub.slots, ub.factor, b, g->stream));
        check_err(g, insert ? "link-cut" : "cut-link");
        g->t_update.launches += nl + 7;
        std::vector<int64_t> part(slots.begin() + c0, slots.begin() + c0 + b);
        for (int64_t x : part) g->h_modified[(size_t)x] = 1;
    }
    refresh_slots(g, slots);
    g->trees_resampled += (int64_t)slots.size();
}

std::vector<int64_t> all_slots(kc_graph *g) {
    std::vector<int64_t> s((size_t)g->pool);
    for (int64_t i = 0; i < g->pool; ++i) s[(size_t)i] = i;
    return s;
}

double weight_sum(kc_graph *g, const std::vector<uint8_t> &flags, int which) {
    UpdBuf ub = upd_buf(g);
    KC_CK(g, cudaMemcpyAsync(ub.flags, flags.data(), flags.size(), cudaMemcpyHostToDevice,
                             g->stream));
    KC_CK(g, launch_weight_sums(g->d_w, ub.flags, g->pool, ub.sums, g->stream));
    double s2[2];
    KC_CK(g, cudaMemcpyAsync(s2, ub.sums, sizeof(s2), cudaMemcpyDeviceToHost, g->stream));
    KC_CK(g, cudaStreamSynchronize(g->stream));
    return which == 2 ? s2[0] + s2[1] : s2[which];
}

void apply_insert(kc_graph *g, int32_t u, int32_t v, int32_t mode, double r_given) {
    {
        UpdPart tp(g->ms_upd_part[0]);
        edit_graph(g, u, v, true);
    }
    // the BIT kernel holds 2m in 32 bits; the scan gives the same f on any graph
    if (g->ttf_variant == KC_TTF_BIT && 2 * g->m >= ((int64_t)1 << 31)) g->ttf_variant = KC_TTF_SCAN;
    double R = r_given;
    if (g->cfg.r_source != KC_R_GIVEN) {
        UpdPart tp(g->ms_upd_part[1]);
        int nl = 0;
        int64_t iters = 0;
        if (!g->d_cg) dalloc(g, &g->d_cg, cg_scratch_doubles(g->n));
        KC_CK(g, resistance_cg(view_of(g), u, v, 1e-13, 50 * g->n + 1000, g->d_cg, &R, &iters,
                               &nl, g->stream, &g->cg_graph));
        g->t_update.launches += nl;
        g->last_cg_iters = iters;
    }
    g->last_r = R;
    UpdPart tp(g->ms_upd_part[2]);
    const int64_t N = g->pool;
    const int64_t k = std::min<int64_t>(N, (int64_t)std::ceil(R * (double)N));
    UpdBuf ub = upd_buf(g);
    std::vector<int64_t> sel((size_t)k);
    if (k > 0) {
        KC_CK(g, launch_select(g->seed, (uint32_t)g->update_seq, N, k, ub.taken, ub.sel, g->stream));
        KC_CK(g, cudaMemcpyAsync(sel.data(), ub.sel, sizeof(int64_t) * k, cudaMemcpyDeviceToHost,
                                 g->stream));
        KC_CK(g, cudaStreamSynchronize(g->stream));
        g->t_update.launches += 1;
    }
    std::sort(sel.begin(), sel.end());
    if (mode == KC_UPDATE_BSM) {
        resample_slots(g, sel, true, u, v);
    } else {
        std::vector<uint8_t> none((size_t)N, 0);
        const double W = weight_sum(g, none, 2);
        transform_slots(g, sel, true, u, v);
        std::vector<uint8_t> flags((size_t)N, 0);
        for (int64_t x : sel) flags[(size_t)x] = 1;
        ub = upd_buf(g);
        KC_CK(g, cudaMemcpyAsync(ub.flags, flags.data(), flags.size(), cudaMemcpyHostToDevice,
                                 g->stream));
        KC_CK(g, launch_weight_rescale(g->d_w, ub.flags, N, ub.sums, R * W, (1.0 - R) * W,
                                       g->stream));
        KC_CK(g, cudaStreamSynchronize(g->stream));
        g->t_update.launches += 2;
    }
    if (g->cfg.refresh_after_update) refresh_slots(g, all_slots(g));
}

void apply_delete(kc_graph *g, int32_t u, int32_t v, int32_t mode) {
    UpdPart tp(g->ms_upd_part[2]);  // the graph edit and tau0 rebuild are moved out below
    const int64_t N = g->pool;
    UpdBuf ub = upd_buf(g);
    KC_CK(g, launch_contains_edge(g->n, N, g->d_parents, u, v, ub.flags, g->stream));
    std::vector<uint8_t> flags((size_t)N, 0);
    KC_CK(g, cudaMemcpyAsync(flags.data(), ub.flags, (size_t)N, cudaMemcpyDeviceToHost, g->stream));
    int32_t pu = 0, pv = 0;
    KC_CK(g, cudaMemcpyAsync(&pu, g->d_p0 + u, sizeof(int32_t), cudaMemcpyDeviceToHost, g->stream));
    KC_CK(g, cudaMemcpyAsync(&pv, g->d_p0 + v, sizeof(int32_t), cudaMemcpyDeviceToHost, g->stream));
    KC_CK(g, cudaStreamSynchronize(g->stream));
    g->t_update.launches += 1;
    std::vector<int64_t> hit;
    for (int64_t i = 0; i < N; ++i)
        if (flags[(size_t)i]) hit.push_back(i);
    const bool tau0_hit = (pu == v) || (pv == u);
    double w_org = 0.0;
    if (mode == KC_UPDATE_ISM) w_org = weight_sum(g, flags, 0);
    const auto tg0 = std::chrono::steady_clock::now();
    edit_graph(g, u, v, false);
    if (tau0_hit) {
        int nl = 0;
        build_tau0(g, nl);
        g->t_update.launches += nl;
        if (f_may_overflow(g->m, g->ecc)) {
            g->last_error = "the rebuilt tau0 is too deep: 4 m^2 ecc(r) >= 2^62";
            throw Fail{KC_ERR_OVERFLOW};
        }
        nl = 0;
        traverse_tau0(g, nl);
        g->t_update.launches += nl;
    }
    {
        const double ms = std::chrono::duration<double, std::milli>(
                              std::chrono::steady_clock::now() - tg0).count();
        g->ms_upd_part[0] += ms;
        g->ms_upd_part[2] -= ms;  // tp adds the whole function at its end
    }
    if (mode == KC_UPDATE_BSM) {
        resample_slots(g, hit, false, u, v);
    } else {
        transform_slots(g, hit, false, u, v);
        ub = upd_buf(g);
        KC_CK(g, cudaMemcpyAsync(ub.flags, flags.data(), flags.size(), cudaMemcpyHostToDevice,
                                 g->stream));
        KC_CK(g, launch_weight_rescale(g->d_w, ub.flags, N, ub.sums, w_org, -1.0, g->stream));
        KC_CK(g, cudaStreamSynchronize(g->stream));
        g->t_update.launches += 2;
    }
    if (g->cfg.refresh_after_update || tau0_hit) refresh_slots(g, all_slots(g));
}

double i128_to_double(long long hi, unsigned long long lo) {
    return std::ldexp((double)hi, 64) + (double)lo;
}

PoolSums reduce_pool(kc_graph *g) {
    PoolSums s{};
    Phase ph(g, g->t_reduce);
    KC_CK(g, launch_pool_reduce(g->d_f, g->d_w, g->pool, 2 * g->m, g->d_scratch, g->stream));
    ph.done(1);
    KC_CK(g, copy_sync(g, &s, g->d_scratch, sizeof(s), cudaMemcpyDeviceToHost));
    return s;
}

// One wave of B trees appended to the pool.
void sample_wave(kc_graph *g, Plan &p, int64_t B, int64_t sid0) {
    run_wave(g, p, B, sid0);
    Carved c = carve(g, p);
    WaveView w = c.wv;
    w.B = B;
    {
        Phase ph(g, g->t_reduce);
        KC_CK(g, launch_pool_append(w, g->pool, g->d_f, g->d_w, g->d_steps, g->d_sid, c.sids,
                                    g->cfg.keep_trees ? g->d_parents : nullptr, g->n,
                                    g->stream));
        ph.done(g->cfg.keep_trees ? 2 : 1);
    }
    for (int64_t k = 0; k < B; ++k) g->h_modified[(size_t)(g->pool + k)] = 0;
    g->pool += B;
    g->last_wave = B;
}

// The autotuner's two pilot waves of B trees each (32 walkers per tree with the
// chunked traversal, then one walker per tree with the leaf-to-root traversal
// where the TTF is the tau0 scan), timed phase by phase without pipelining;
// the faster walker and traversal are kept.  The trees are the same either way.
void autotune(kc_graph *g, Plan &p, int64_t B, int64_t sid0) {
    g->tuning = true;
    const bool scan = g->ttf_variant == KC_TTF_SCAN;
    const int modes[2] = {kTravChunked, scan ? kTravLeafUp : kTravChunked};
    const int walkers[2] = {KC_WALK_WARP, KC_WALK_LANE};
    double wms[2], tms[2];
    try {
        for (int k = 0; k < 2; ++k) {
            g->walker = walkers[k];
            g->trav_mode = modes[k];
            const double w0 = g->t_wilson.ms, t0 = g->t_traverse.ms;
            sample_wave(g, p, B, sid0 + k * B);
            wms[k] = (g->t_wilson.ms - w0) / (double)B;
            tms[k] = (g->t_traverse.ms - t0) / (double)B;
        }
    } catch (Fail &) {
        g->tuning = false;
        g->walker = KC_WALK_WARP;
        g->trav_mode = -1;
        throw;
    }
    g->tuning = false;
    g->walker = wms[1] < wms[0] ? KC_WALK_LANE : KC_WALK_WARP;
    g->trav_mode = (scan && tms[1] < tms[0]) ? kTravLeafUp : kTravChunked;
    g->tune_ms[0] = wms[0];
    g->tune_ms[1] = wms[1];
    g->tune_ms[2] = tms[0];
    g->tune_ms[3] = scan ? tms[1] : 0.0;
    g->tuned = true;
}

// Rejection by walk length, one wave of B trees from sample id sid0 without
// pipelining: the walk, then the accepted trees' traversal and f through a
// tree map.  Leaves steps (-1: rejected) and f in the carved workspace.
void run_wave_reject(kc_graph *g, Plan &p, int64_t B, int64_t sid0) {
    const GraphView gv = view_of(g);
    Carved c = carve(g, p);
    WaveView w = c.wv;
    w.B = B;
    KC_CK(g, cudaMemsetAsync(g->d_err, 0, 2 * sizeof(uint32_t), g->stream));
    KC_CK(g, cudaMemsetAsync(w.f, 0, sizeof(int64_t) * (size_t)B, g->stream));
    KC_CK(g, launch_iota(c.sids, sid0, B, g->stream));
    reset_segtab(g, B);
    {
        Phase ph(g, g->t_init);
        KC_CK(g, launch_wave_init(gv, w, g->stream));
        ph.done(1);
    }
    {
        Phase ph(g, g->t_wilson);
        if (g->walker == KC_WALK_LANE)
            KC_CK(g, launch_wilson_reject(gv, w, g->seed, c.sids, nullptr, g->cfg.reject_steps,
                                          g->stream));
        else
            KC_CK(g, launch_wilson_warp_reject(gv, w, g->seed, c.sids, g->d_sorder,
                                               g->cfg.reject_steps, g->stream));
        ph.done(1);
    }
    uint32_t hdr[2] = {0, 0};
    KC_CK(g, copy_sync(g, hdr, g->d_err, sizeof(hdr), cudaMemcpyDeviceToHost));
    if (hdr[0] & kErrStepLimit) {
        // a single vertex's departure counter filled its 25 bits
        g->last_error = "Wilson walk exceeded the per-vertex departure limit";
        throw Fail{KC_ERR_STEP_LIMIT};
    }
    if (hdr[0]) {
        g->last_error = "Wilson walkers reached an inconsistent state or the iteration cap";
        throw Fail{KC_ERR_CUDA};
    }
    std::vector<int64_t> st((size_t)B);
    KC_CK(g, copy_sync(g, st.data(), w.steps, sizeof(int64_t) * (size_t)B,
                       cudaMemcpyDeviceToHost));
    int64_t na = 0;
    std::vector<SegRegion> spare;  // walk arrays of the rejected trees
    for (int64_t t = 0; t < B; ++t) {
        if (st[(size_t)t] >= 0) {
            g->h_map[na++] = (int32_t)t;
        } else {
            spare.push_back({(uintptr_t)(w.word + t * g->n), sizeof(uint64_t) * (size_t)g->n});
            spare.push_back({(uintptr_t)(w.ord + t * g->n), sizeof(int32_t) * (size_t)g->n});
        }
    }
    if (na == 0) return;
    KC_CK(g, cudaMemcpyAsync(g->d_map, g->h_map, sizeof(int32_t) * (size_t)na,
                             cudaMemcpyHostToDevice, g->stream));
    if (p.bit) {
        ensure_stack(g, p, hdr[1]);
        c = carve(g, p);
    }
    for (int64_t off = 0; off < na; off += p.BT) {
        WaveView sv = c.wv;
        sv.B = std::min<int64_t>(p.BT, na - off);
        sv.tmap = g->d_map + off;
        {
            Phase ph(g, g->t_traverse);
            int nl = 0;
            KC_CK(g, launch_traverse(gv, sv, p.bit, g->stream, &nl, fast_traversal(g)));
            ph.done(nl);
        }
        {
            Phase ph(g, g->t_ttf);
            int nl = 1;
            if (p.bit) nl = eval_ttf_bit(g, gv, p, sv, true, spare, g->stream);
            else KC_CK(g, launch_ttf_scan(gv, sv, g->stream));
            ph.done(nl);
        }
    }
    KC_CK(g, copy_sync(g, hdr, g->d_err, sizeof(hdr), cudaMemcpyDeviceToHost));
    if (hdr[0] & kErrBadTree) {
        g->last_error = "inconsistent tree state or traversal stack overflow";
        throw Fail{KC_ERR_CUDA};
    }
}

// Rejection by walk length: waves of the 32-walker kernel abandon trees past
// cfg.reject_steps departures; each wave's accepted trees are traversed and
// evaluated (overlapping the walk, as pipelined waves do, on large graphs) and
// appended to the pool in sample-id order, until ntrees are accepted.
// A wave draws about need / rate trees, rate being the acceptance rate seen on
// this handle so far (before any is seen: cfg.reject_accept_hint, else 8/9), so that one
// wave usually suffices; of its accepted trees only the first `need` in id
// order are kept, and the ids after the last kept one are left for the next
// call.  Rejected ids below it are consumed (never reused).
void do_sample_reject(kc_graph *g, int64_t ntrees) {
    const double hint = g->cfg.reject_accept_hint > 0 ? g->cfg.reject_accept_hint : 8.0 / 9.0;
    auto wave_size = [&](int64_t need) {
        return kc_host::reject_wave_size(need, g->rej_drawn, g->rej_accepted, hint);
    };
    ensure_pool(g, g->pool + ntrees);
    // the wave's accepted trees stream through traversal chunks, so the walk
    // may take most of the budget: with one walker per tree, every tree of a
    // wave walks at once and a wave lasts about reject_steps departures
    Plan p = plan_for(g, wave_size(ntrees), false, 0.9);
    ensure_ws(g, p);
    ensure_pipeline(g, p.BW);  // done flags and tree-map staging
    const int64_t pool0 = g->pool, sid_base = g->next_sid, rej0 = g->trees_rejected;
    const int64_t drawn0 = g->rej_drawn, acc0 = g->rej_accepted;
    try {
        int64_t accepted = 0;
        while (accepted < ntrees) {
            if (g->next_sid - sid_base > 64 * ntrees + 4096) {
                g->last_error = "rejection by walk length accepts too few trees: raise reject_steps";
                throw Fail{KC_ERR_STEP_LIMIT};
            }
            const int64_t need = ntrees - accepted;
            int64_t B = std::min<int64_t>(p.BW, wave_size(need));
            B = std::min<int64_t>(B, ((int64_t)1 << 32) - g->next_sid);
            if (B <= 0) {
                g->last_error = "kc_sample: sample ids must stay below 2^32";
                throw Fail{KC_ERR_INVALID_ARG};
            }
            if (B > 1 && (B > p.BT || g->n >= (1 << 16))) {
                try {
                    run_wave_pipelined(g, p, B, g->next_sid, true);
                } catch (Fail &) {
                    // let both streams drain before the workspace is reused
                    cudaStreamSynchronize(g->stream);
                    if (g->stream2) cudaStreamSynchronize(g->stream2);
                    throw;
                }
            } else {
                run_wave_reject(g, p, B, g->next_sid);
            }
            const WaveView w = carve(g, p).wv;
            std::vector<int64_t> st((size_t)B), f((size_t)B);
            KC_CK(g, copy_sync(g, st.data(), w.steps, sizeof(int64_t) * (size_t)B,
                               cudaMemcpyDeviceToHost));
            KC_CK(g, copy_sync(g, f.data(), w.f, sizeof(int64_t) * (size_t)B,
                               cudaMemcpyDeviceToHost));
            std::vector<int64_t> af, as, ai;
            int64_t used = B, wave_acc = 0;  // ids consumed; accepted in the whole wave
            for (int64_t t = 0; t < B; ++t) {
                if (st[(size_t)t] < 0) continue;
                ++wave_acc;
                if ((int64_t)af.size() == need) continue;
                af.push_back(f[(size_t)t]);
                as.push_back(st[(size_t)t]);
                ai.push_back(g->next_sid + t);
                if ((int64_t)af.size() == need) used = t + 1;
            }
            const int64_t na = (int64_t)af.size();
            if (na > 0) {
                std::vector<double> aw((size_t)na, 1.0);
                const size_t b8 = sizeof(int64_t) * (size_t)na;
                KC_CK(g, cudaMemcpyAsync(g->d_f + g->pool, af.data(), b8, cudaMemcpyHostToDevice,
                                         g->stream));
                KC_CK(g, cudaMemcpyAsync(g->d_steps + g->pool, as.data(), b8,
                                         cudaMemcpyHostToDevice, g->stream));
                KC_CK(g, cudaMemcpyAsync(g->d_sid + g->pool, ai.data(), b8, cudaMemcpyHostToDevice,
                                         g->stream));
                KC_CK(g, cudaMemcpyAsync(g->d_w + g->pool, aw.data(), sizeof(double) * (size_t)na,
                                         cudaMemcpyHostToDevice, g->stream));
                KC_CK(g, cudaStreamSynchronize(g->stream));
                for (int64_t k = 0; k < na; ++k) g->h_modified[(size_t)(g->pool + k)] = 0;
                g->pool += na;
            }
            g->last_wave = B;
            g->trees_rejected += used - na;
            g->next_sid += used;
            g->rej_drawn += B;
            g->rej_accepted += wave_acc;
            accepted += na;
        }
    } catch (Fail &) {
        g->pool = pool0;
        g->next_sid = sid_base;
        g->trees_rejected = rej0;
        g->rej_drawn = drawn0;
        g->rej_accepted = acc0;
        throw;
    }
}

void do_sample(kc_graph *g, int64_t ntrees) {
    if (ntrees <= 0) return;
    if (g->cfg.reject_steps > 0) {
        do_sample_reject(g, ntrees);
        return;
    }
    ensure_pool(g, g->pool + ntrees);
    Plan p = plan_for(g, ntrees, false);
    ensure_ws(g, p);
    const int64_t pool0 = g->pool, sid_base = g->next_sid;
    int64_t done = 0;
    if (g->cfg.autotune && !g->tuned && ntrees >= 64) {
        const int64_t B = std::min<int64_t>(p.BW, ntrees / 2);
        try {
            autotune(g, p, B, sid_base);
        } catch (Fail &) {
            g->pool = pool0;
            g->next_sid = sid_base;
            throw;
        }
        done = 2 * B;
    }
    try {
        // equal waves: a short last wave would take as long as a full one
        const int64_t rest = ntrees - done;
        const int64_t waves = (rest + p.BW - 1) / p.BW;
        const int64_t per_wave = waves > 0 ? (rest + waves - 1) / waves : 0;
        while (done < ntrees) {
            const int64_t B = std::min<int64_t>(per_wave, ntrees - done);
            sample_wave(g, p, B, sid_base + done);
            done += B;
        }
    } catch (Fail &) {
        g->pool = pool0;
        g->next_sid = sid_base;
        throw;
    }
    g->next_sid = sid_base + ntrees;
}

// Batched multi-graph sampling: the walks of every graph's wave run in one
// 32-walker launch (one warp per tree, graphs mixed), then each graph's
// traversal, TTF and pool append.  All work goes to the first graph's stream.
void do_sample_multi(kc_graph *const *gs, const int64_t *n_trees, int32_t count) {
    cudaStream_t s0 = gs[0]->stream;
    std::vector<cudaStream_t> saved((size_t)count);
    std::vector<int64_t> pool0((size_t)count), sid0((size_t)count), left((size_t)count);
    std::vector<Plan> plans((size_t)count);
    for (int32_t i = 0; i < count; ++i) {
        kc_graph *g = gs[i];
        saved[(size_t)i] = g->stream;
        g->stream = s0;
        pool0[(size_t)i] = g->pool;
        sid0[(size_t)i] = g->next_sid;
        left[(size_t)i] = n_trees[i];
    }
    void *d_tab = nullptr;
    try {
        for (int32_t i = 0; i < count; ++i) {
            kc_graph *g = gs[i];
            if (n_trees[i] <= 0) continue;
            ensure_pool(g, g->pool + n_trees[i]);
            plans[(size_t)i] = plan_for(g, n_trees[i], false);
            ensure_ws(g, plans[(size_t)i]);
        }
        for (;;) {
            // this pass: up to one wave per graph
            std::vector<GraphView> gv;
            std::vector<WaveView> wv;
            std::vector<uint64_t> seeds;
            std::vector<const int64_t *> sids;
            std::vector<const int32_t *> sorders;
            std::vector<int64_t> caps;
            std::vector<int32_t> idx;  // graph of each table row
            std::vector<int64_t> bs;
            for (int32_t i = 0; i < count; ++i) {
                kc_graph *g = gs[i];
                if (left[(size_t)i] <= 0) continue;
                const int64_t B = std::min<int64_t>(left[(size_t)i], plans[(size_t)i].BW);
                Carved c = carve(g, plans[(size_t)i]);
                WaveView w = c.wv;
                w.B = B;
                const GraphView v = view_of(g);
                KC_CK(g, cudaMemsetAsync(g->d_err, 0, 2 * sizeof(uint32_t), s0));
                KC_CK(g, launch_iota(c.sids, g->next_sid, B, s0));
                KC_CK(g, launch_wave_init(v, w, s0));
                gv.push_back(v);
                wv.push_back(w);
                seeds.push_back(g->seed);
                sids.push_back(c.sids);
                sorders.push_back(g->d_sorder);
                caps.push_back(step_cap_of(g));
                idx.push_back(i);
                bs.push_back(B);
            }
            if (idx.empty()) break;
            const size_t G = idx.size();
            // trees of different graphs interleaved, so a launch mixes sizes
            std::vector<int2> entry;
            int64_t most = 0;
            for (int64_t b : bs) most = std::max(most, b);
            for (int64_t t = 0; t < most; ++t)
                for (size_t k = 0; k < G; ++k)
                    if (t < bs[k]) entry.push_back(make_int2((int)k, (int)t));
            const size_t bytes = sizeof(GraphView) * G + sizeof(WaveView) * G + 8 * G * 4 +
                                 sizeof(int2) * entry.size() + 256 * 8;
            kc_graph *g0 = gs[0];
            KC_CK(g0, cudaMallocAsync(&d_tab, bytes, s0));
            char *base = (char *)d_tab;
            size_t off = 0;
            auto put = [&](const void *src, size_t nb) {
                void *dst = base + off;
                KC_CK(g0, cudaMemcpyAsync(dst, src, nb, cudaMemcpyHostToDevice, s0));
                off += (nb + 255) & ~size_t(255);
                return dst;
            };
            MultiWalk mw;
            mw.graphs = (const GraphView *)put(gv.data(), sizeof(GraphView) * G);
            mw.waves = (const WaveView *)put(wv.data(), sizeof(WaveView) * G);
            mw.seeds = (const uint64_t *)put(seeds.data(), 8 * G);
            mw.sids = (const int64_t *const *)put(sids.data(), 8 * G);
            mw.sorders = (const int32_t *const *)put(sorders.data(), 8 * G);
            mw.step_caps = (const int64_t *)put(caps.data(), 8 * G);
            mw.entry = (const int2 *)put(entry.data(), sizeof(int2) * entry.size());
            mw.count = (int64_t)entry.size();
            {
                Phase ph(g0, g0->t_wilson);
                KC_CK(g0, launch_wilson_warp_multi(mw, s0));
                ph.done(1);
            }
            KC_CK(g0, cudaFreeAsync(d_tab, s0));
            d_tab = nullptr;
            // per graph: walk errors, BIT stacks, sub-wave buffers zeroed; the
            // graphs whose wave is one sub-wave get one batched traversal and TTF
            // launch, the others their own launches
            std::vector<Carved> cv(G);
            std::vector<GraphView> tg;
            std::vector<WaveView> tw;
            std::vector<int2> e_all, e_scan, e_bit;
            int64_t max_n = 0;
            for (size_t k = 0; k < G; ++k) {
                const int32_t i = idx[k];
                kc_graph *g = gs[i];
                Plan &p = plans[(size_t)i];
                const int64_t B = bs[k];
                uint32_t hdr[2] = {0, 0};
                KC_CK(g, copy_sync(g, hdr, g->d_err, sizeof(hdr), cudaMemcpyDeviceToHost));
                if (hdr[0] & kErrStepLimit) {
                    g->last_error = "Wilson walk exceeded the step cap";
                    throw Fail{KC_ERR_STEP_LIMIT};
                }
                if (hdr[0]) throw Fail{KC_ERR_CUDA};
                if (p.bit) ensure_stack(g, p, hdr[1]);
                cv[k] = carve(g, p);
                WaveView w = cv[k].wv;
                w.B = B;
                const GraphView v = view_of(g);
                if (B <= p.BT) {
                    const size_t nb = (size_t)B * (size_t)g->n;
                    KC_CK(g, cudaMemsetAsync(w.size, 0, sizeof(int32_t) * nb, s0));
                    KC_CK(g, cudaMemsetAsync(w.vol, 0, sizeof(int64_t) * nb, s0));
                    if (p.bit) {
                        KC_CK(g, cudaMemsetAsync(w.bit, 0,
                                                 sizeof(int64_t) * (size_t)B * (size_t)(g->n + 1),
                                                 s0));
                    } else {
                        KC_CK(g, cudaMemsetAsync(w.f, 0, sizeof(int64_t) * (size_t)B, s0));
                        w.bit = nullptr;
                    }
                    const int gk = (int)tg.size();
                    tg.push_back(v);
                    tw.push_back(w);
                    for (int64_t t = 0; t < B; ++t) {
                        e_all.push_back(make_int2(gk, (int)t));
                        (p.bit ? e_bit : e_scan).push_back(make_int2(gk, (int)t));
                    }
                    max_n = std::max<int64_t>(max_n, g->n);
                    g->t_traverse.launches += 2;
                    g->t_ttf.launches += 1;
                    continue;
                }
                for (int64_t sub = 0; sub < B; sub += p.BT) {
                    const int64_t b = std::min<int64_t>(p.BT, B - sub);
                    WaveView sw = w;
                    sw.B = b;
                    sw.word = w.word + sub * g->n;
                    sw.ord = w.ord + sub * g->n;
                    sw.steps = w.steps + sub;
                    sw.f = w.f + sub;
                    int nl = 0;
                    KC_CK(g, launch_traverse(v, sw, p.bit, s0, &nl, fast_traversal(g)));
                    if (p.bit) KC_CK(g, launch_ttf_bit(v, sw, s0));
                    else KC_CK(g, launch_ttf_scan(v, sw, s0));
                    g->t_traverse.launches += nl;
                    g->t_ttf.launches += 1;
                }
            }
            if (!tg.empty()) {
                const size_t Gt = tg.size();
                const size_t tb = sizeof(GraphView) * Gt + sizeof(WaveView) * Gt +
                                  sizeof(int2) * (e_all.size() + e_scan.size() + e_bit.size()) +
                                  256 * 6;
                KC_CK(g0, cudaMallocAsync(&d_tab, tb, s0));
                char *tbase = (char *)d_tab;
                size_t toff = 0;
                auto tput = [&](const void *src, size_t nb) {
                    void *dst = tbase + toff;
                    if (nb) KC_CK(g0, cudaMemcpyAsync(dst, src, nb, cudaMemcpyHostToDevice, s0));
                    toff += (nb + 255) & ~size_t(255);
                    return dst;
                };
                MultiSub ms;
                ms.graphs = (const GraphView *)tput(tg.data(), sizeof(GraphView) * Gt);
                ms.waves = (const WaveView *)tput(tw.data(), sizeof(WaveView) * Gt);
                MultiSub m_all = ms, m_scan = ms, m_bit = ms;
                m_all.entry = (const int2 *)tput(e_all.data(), sizeof(int2) * e_all.size());
                m_all.count = (int64_t)e_all.size();
                m_scan.entry = (const int2 *)tput(e_scan.data(), sizeof(int2) * e_scan.size());
                m_scan.count = (int64_t)e_scan.size();
                m_bit.entry = (const int2 *)tput(e_bit.data(), sizeof(int2) * e_bit.size());
                m_bit.count = (int64_t)e_bit.size();
                KC_CK(g0, launch_traverse_multi(m_all, s0));
                KC_CK(g0, launch_ttf_scan_multi(m_scan, max_n, s0));
                KC_CK(g0, launch_ttf_bit_multi(m_bit, s0));
                KC_CK(g0, cudaFreeAsync(d_tab, s0));
                d_tab = nullptr;
            }
            for (size_t k = 0; k < G; ++k) {
                const int32_t i = idx[k];
                kc_graph *g = gs[i];
                const int64_t B = bs[k];
                WaveView w = cv[k].wv;
                w.B = B;
                KC_CK(g, launch_pool_append(w, g->pool, g->d_f, g->d_w, g->d_steps, g->d_sid,
                                            cv[k].sids, g->cfg.keep_trees ? g->d_parents : nullptr,
                                            g->n, s0));
                uint32_t hdr[2] = {0, 0};
                KC_CK(g, copy_sync(g, hdr, g->d_err, sizeof(hdr), cudaMemcpyDeviceToHost));
                if (hdr[0]) throw Fail{KC_ERR_CUDA};
                for (int64_t q = 0; q < B; ++q) g->h_modified[(size_t)(g->pool + q)] = 0;
                g->pool += B;
                g->next_sid += B;
                g->last_wave = B;
                left[(size_t)i] -= B;
            }
        }
    } catch (Fail &) {
        if (d_tab) cudaFreeAsync(d_tab, s0);
        cudaStreamSynchronize(s0);
        for (int32_t i = 0; i < count; ++i) {
            gs[i]->pool = pool0[(size_t)i];
            gs[i]->next_sid = sid0[(size_t)i];
            gs[i]->stream = saved[(size_t)i];
        }
        throw;
    }
    for (int32_t i = 0; i < count; ++i) gs[i]->stream = saved[(size_t)i];
}

}  // namespace

// =========================================================================
// C ABI
// =========================================================================
extern "C" {

void kc_config_default(kc_config *cfg) {
    if (!cfg) return;
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->struct_size = sizeof(kc_config);
    cfg->root = -1;
    cfg->ttf_variant = KC_TTF_AUTO;
    cfg->keep_trees = 1;
    cfg->stop_rule = KC_STOP_CLT;
    cfg->refresh_after_update = 0;
    cfg->inputs_on_device = 0;
    cfg->r_source = KC_R_CG;
    cfg->max_trees_in_flight = 0;
    cfg->batch_trees = 1024;
    cfg->max_trees = (int64_t)1 << 24;
    cfg->step_cap = 0;
    cfg->mem_fraction = 0.8;
}

const char *kc_status_string(kc_status s) {
    switch (s) {
        case KC_OK: return "ok";
        case KC_ERR_INVALID_ARG: return "invalid argument";
        case KC_ERR_NOT_SYMMETRIC: return "graph is not symmetric";
        case KC_ERR_SELF_LOOP: return "graph has a self loop";
        case KC_ERR_MULTI_EDGE: return "row not strictly ascending (repeated edge or unsorted)";
        case KC_ERR_DISCONNECTED: return "graph is disconnected";
        case KC_ERR_OVERFLOW: return "4 m^2 ecc(r) >= 2^62: f(tau) may overflow int64";
        case KC_ERR_OUT_OF_MEMORY: return "device out of memory";
        case KC_ERR_CUDA: return "CUDA error";
        case KC_ERR_STEP_LIMIT: return "Wilson walk exceeded the step cap";
        case KC_ERR_EDGE_EXISTS: return "inserted edge already exists";
        case KC_ERR_EDGE_MISSING: return "deleted edge does not exist";
        case KC_ERR_BRIDGE: return "deleted edge is a bridge";
        case KC_ERR_NO_SAMPLES: return "no sampled trees";
        case KC_ERR_NO_DEVICE: return "no sm_103 CUDA device";
        case KC_ERR_NOT_RETAINED: return "trees were not retained (keep_trees = 0)";
        case KC_ERR_SCRATCH_LIMIT:
            return "request exceeds the 8 Mi-word (64 MiB) fixed scratch of kc_wilson_noalloc";
    }
    return "unknown status";
}

const char *kc_last_error(kc_graph *g) { return g ? g->last_error.c_str() : ""; }

kc_status kc_graph_destroy(kc_graph *g) {
    if (!g) return KC_OK;
    dfree(g->d_row_off);
    dfree(g->d_col);
    dfree(g->d_deg);
    dfree(g->d_rec);
    dfree(g->d_p0);
    dfree(g->d_level0);
    dfree(g->d_in0);
    dfree(g->d_out0);
    dfree(g->d_f);
    dfree(g->d_w);
    dfree(g->d_steps);
    dfree(g->d_sid);
    dfree(g->d_parents);
    dfree(g->d_ws);
    if (g->d_ub) cudaFree(g->d_ub);
    dfree(g->d_edit);
    dfree(g->d_cg);
    cg_graph_release(g->cg_graph);
    dfree(g->d_stack);
    dfree(g->d_sorder);
    dfree(g->d_err);
    if (g->d_scratch) cudaFree(g->d_scratch);
    hfree(g->h_done);
    hfree(g->h_map);
    hfree(g->h_segtab);
    dfree(g->d_segtab);
    dfree(g->d_segx);
    dfree(g->d_map);
    if (g->stream2) cudaStreamDestroy(g->stream2);
    if (g->ev0) cudaEventDestroy(g->ev0);
    if (g->ev1) cudaEventDestroy(g->ev1);
    delete g;
    clear_stale_error();  // nothing the frees above report outlives this call
    return KC_OK;
}

kc_status kc_graph_create(int64_t n, const int64_t *row_off, const int32_t *col,
                          const kc_config *cfg_in, kc_graph **out) {
    if (!out) return KC_ERR_INVALID_ARG;
    *out = nullptr;
    if (n < 2 || !row_off || !col) return KC_ERR_INVALID_ARG;
    if (n > (int64_t)0x7FFFFFFF - 1) return KC_ERR_INVALID_ARG;
    kc_config cfg;
    kc_config_default(&cfg);
    if (cfg_in) {
        if (cfg_in->struct_size != sizeof(kc_config)) return KC_ERR_INVALID_ARG;
        cfg = *cfg_in;
    }
    if (cfg.walker < KC_WALK_AUTO || cfg.walker > KC_WALK_HYBRID ||
        cfg.hybrid_prefix_permille < 0 || cfg.hybrid_tail_permille < 0 ||
        cfg.tau0_kind < KC_TAU0_BFS || cfg.tau0_kind > KC_TAU0_WILSON)
        return KC_ERR_INVALID_ARG;
    // rejection by walk length: the 32-walker kernel, static pools, and a cap a
    // tree can meet (every non-root vertex departs at least once)
    if (!(cfg.reject_accept_hint >= 0 && cfg.reject_accept_hint <= 1)) return KC_ERR_INVALID_ARG;
    if (cfg.ttf_segments < 0 || cfg.ttf_segments > 64) return KC_ERR_INVALID_ARG;
    if (cfg.reject_steps < 0 ||
        (cfg.reject_steps > 0 &&
         (cfg.reject_steps < n - 1 || cfg.keep_trees || cfg.autotune ||
          cfg.walker == KC_WALK_HYBRID)))
        return KC_ERR_INVALID_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        (void)cudaGetLastError();
        return KC_ERR_NO_DEVICE;
    }
    kc_graph *g = new (std::nothrow) kc_graph();
    if (!g) return KC_ERR_OUT_OF_MEMORY;
    g->cfg = cfg;
    try {
        clear_stale_error();
        KC_CK(g, cudaGetDevice(&g->device));
        cudaDeviceProp prop;
        KC_CK(g, cudaGetDeviceProperties(&prop, g->device));
        if (prop.major != 10 || prop.minor != 3) {
            g->last_error = "the library is built for sm_103a only";
            throw Fail{KC_ERR_NO_DEVICE};
        }
        g->resident_trees = (int64_t)prop.multiProcessorCount * wilson_warp_blocks_per_sm();
        g->num_sms = prop.multiProcessorCount;
        KC_CK(g, cudaEventCreate(&g->ev0));
        KC_CK(g, cudaEventCreate(&g->ev1));
        g->n = n;
        if (cfg.sample_id_base < 0 || cfg.sample_id_base >= ((int64_t)1 << 32))
            throw Fail{KC_ERR_INVALID_ARG};
        g->next_sid = cfg.sample_id_base;
        // host copy of the CSR (validated layout, kept for updates)
        g->h_row_off.resize((size_t)n + 1);
        const cudaMemcpyKind kind = cfg.inputs_on_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost;
        KC_CK(g, copy_sync(g, g->h_row_off.data(), row_off, sizeof(int64_t) * (n + 1), kind));
        if (g->h_row_off[0] != 0) throw Fail{KC_ERR_INVALID_ARG};
        for (int64_t v = 0; v < n; ++v)
            if (g->h_row_off[v + 1] < g->h_row_off[v]) throw Fail{KC_ERR_INVALID_ARG};
        const int64_t twom = g->h_row_off[n];
        if (twom % 2 != 0 || twom == 0) throw Fail{twom == 0 ? KC_ERR_DISCONNECTED : KC_ERR_NOT_SYMMETRIC};
        g->m = twom / 2;
        g->h_col.resize((size_t)twom);
        KC_CK(g, copy_sync(g, g->h_col.data(), col, sizeof(int32_t) * twom, kind));

        dalloc(g, &g->d_row_off, n + 1);
        dalloc(g, &g->d_col, twom);
        g->col_cap = (size_t)twom;
        dalloc(g, &g->d_deg, n);
        dalloc(g, &g->d_rec, n);
        dalloc(g, &g->d_p0, n);
        dalloc(g, &g->d_level0, n);
        dalloc(g, &g->d_in0, n);
        dalloc(g, &g->d_out0, n);
        dalloc(g, &g->d_err, 4);
        g->scratch_bytes = 4096;
        KC_CK(g, cudaMalloc(&g->d_scratch, g->scratch_bytes));
        KC_CK(g, cudaMemcpyAsync(g->d_row_off, g->h_row_off.data(), sizeof(int64_t) * (n + 1),
                                 cudaMemcpyHostToDevice, g->stream));
        KC_CK(g, cudaMemcpyAsync(g->d_col, g->h_col.data(), sizeof(int32_t) * twom,
                                 cudaMemcpyHostToDevice, g->stream));

        Phase ph(g, g->t_setup);
        int launches = 0;
        GraphView gv = view_of(g);
        KC_CK(g, launch_build_records(gv, g->d_rec, g->d_deg, g->stream));
        ++launches;
        uint32_t *d_flags = g->d_err;
        KC_CK(g, cudaMemsetAsync(d_flags, 0, 4 * sizeof(uint32_t), g->stream));
        KC_CK(g, launch_validate(gv, d_flags, g->stream));
        ++launches;
        uint32_t flags = 0;
        KC_CK(g, cudaMemcpyAsync(&flags, d_flags, sizeof(flags), cudaMemcpyDeviceToHost, g->stream));
        KC_CK(g, cudaStreamSynchronize(g->stream));
        if (flags & 1u) throw Fail{KC_ERR_INVALID_ARG};
        if (flags & 2u) throw Fail{KC_ERR_SELF_LOOP};
        if (flags & 4u) throw Fail{KC_ERR_MULTI_EDGE};
        if (flags & 8u) throw Fail{KC_ERR_NOT_SYMMETRIC};
        if (flags & 16u) throw Fail{KC_ERR_DISCONNECTED};

        // root
        if (cfg.root >= 0) {
            if (cfg.root >= n) throw Fail{KC_ERR_INVALID_ARG};
            g->root = cfg.root;
        } else {
            unsigned long long *d_best = (unsigned long long *)g->d_scratch;
            KC_CK(g, cudaMemsetAsync(d_best, 0, sizeof(unsigned long long), g->stream));
            KC_CK(g, launch_root(gv, d_best, g->stream));
            ++launches;
            unsigned long long best = 0;
            KC_CK(g, cudaMemcpyAsync(&best, d_best, sizeof(best), cudaMemcpyDeviceToHost, g->stream));
            KC_CK(g, cudaStreamSynchronize(g->stream));
            g->root = (int32_t)(0xFFFFFFFFull - (best & 0xFFFFFFFFull));
            if (cfg.root == -1) g->root = central_root(g, g->root, launches);
        }
        gv.root = g->root;
        // Start order of the concurrent walkers: a fixed pseudo-random
        // permutation (vertices sorted by a 32-bit mix of their id), so that the
        // 32 walkers of a tree start far apart and rarely block each other.  Any
        // order gives the same trees; starting walkers next to each other (for
        // example in BFS order around the root) makes them collide constantly.
        {
            std::vector<uint64_t> key((size_t)n);
            for (int64_t v = 0; v < n; ++v) {
                uint32_t h = (uint32_t)v * 0x9E3779B1u;
                h ^= h >> 15;
                h *= 0x85EBCA77u;
                h ^= h >> 13;
                h *= 0xC2B2AE3Du;
                h ^= h >> 16;
                key[(size_t)v] = ((uint64_t)h << 32) | (uint64_t)(uint32_t)v;
            }
            std::vector<int32_t> order((size_t)n);
            for (int64_t v = 0; v < n; ++v) order[(size_t)v] = (int32_t)v;
            std::sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
                return key[(size_t)a] < key[(size_t)b] || (key[(size_t)a] == key[(size_t)b] && a < b);
            });
            dalloc(g, &g->d_sorder, n);
            KC_CK(g, cudaMemcpyAsync(g->d_sorder, order.data(), sizeof(int32_t) * n,
                                     cudaMemcpyHostToDevice, g->stream));
            KC_CK(g, cudaStreamSynchronize(g->stream));
        }
        build_tau0(g, launches);
        gv.ecc = g->ecc;

        if (f_may_overflow(g->m, g->ecc)) throw Fail{KC_ERR_OVERFLOW};
        traverse_tau0(g, launches);
        ph.done(launches);
        // TTF variant (Theorem 8: O(n min(Delta, log n)))
        int lg = 0;
        while (((int64_t)1 << lg) < n) ++lg;
        int variant = cfg.ttf_variant;
        if (variant == KC_TTF_AUTO) variant = (g->ecc <= 2 * lg) ? KC_TTF_SCAN : KC_TTF_BIT;
        if (variant == KC_TTF_BIT && twom >= ((int64_t)1 << 31)) variant = KC_TTF_SCAN;
        g->ttf_variant = variant;
        // Walkers: one sequential walker per tree leaves the GPU nearly idle
        // whenever fewer trees fit in memory than it has warp slots, and a wave
        // lasts as long as its slowest tree; 32 walkers per tree finish the
        // long trees of road-shaped graphs about 4 steps per iteration, so they
        // are the default.  Under rejection by walk length on a long-diameter
        // graph (BIT variant) no tree walks past the cap, and one walker per
        // tree keeps every tree of the wave in flight from the start (32-walker
        // trees wait for one of the SMs' warp slots): the wave then lasts about
        // cap x one walker's time per departure, which measured shorter.
        int walker = cfg.walker;
        if (walker == KC_WALK_AUTO || cfg.autotune)
            walker = (cfg.reject_steps > 0 && !cfg.autotune && variant == KC_TTF_BIT)
                         ? KC_WALK_LANE : KC_WALK_WARP;
        g->walker = walker;
    } catch (Fail &f) {
        kc_graph_destroy(g);
        return f.st;
    }
    *out = g;
    return KC_OK;
}

kc_status kc_graph_set_workspace_limit(kc_graph *g, int64_t bytes) {
    if (!g || bytes < 0) return KC_ERR_INVALID_ARG;
    g->ws_limit = bytes;
    return KC_OK;
}

kc_status kc_graph_release_workspace(kc_graph *g) {
    if (!g) return KC_ERR_INVALID_ARG;
    try {
        clear_stale_error();
        release_ws(g);
    } catch (Fail &f) {
        return f.st;
    }
    return KC_OK;
}

kc_status kc_graph_reset(kc_graph *g, uint64_t seed, int64_t sample_id_base) {
    if (!g || sample_id_base < 0 || sample_id_base >= ((int64_t)1 << 32))
        return KC_ERR_INVALID_ARG;
    g->pool = 0;
    g->next_sid = sample_id_base;
    g->seed = seed;
    g->seeded = true;
    g->last_wave = 0;
    return KC_OK;
}

kc_status kc_graph_set_stream(kc_graph *g, void *cuda_stream) {
    if (!g) return KC_ERR_INVALID_ARG;
    g->stream = (cudaStream_t)cuda_stream;
    return KC_OK;
}

kc_status kc_sample(kc_graph *g, uint64_t seed, int64_t n_trees) {
    if (!g || n_trees < 0) return KC_ERR_INVALID_ARG;
    if (g->seeded && seed != g->seed) {
        g->last_error = "kc_sample: the handle is already seeded with a different seed";
        return KC_ERR_INVALID_ARG;
    }
    if (n_trees == 0) return KC_OK;
    if (g->next_sid + n_trees > ((int64_t)1 << 32)) {
        g->last_error = "kc_sample: sample ids must stay below 2^32";
        return KC_ERR_INVALID_ARG;
    }
    const bool was_seeded = g->seeded;
    g->seed = seed;
    g->seeded = true;
    try {
        clear_stale_error();
        do_sample(g, n_trees);
    } catch (Fail &f) {
        g->seeded = was_seeded;
        return f.st;
    }
    return KC_OK;
}

kc_status kc_reserve(kc_graph *g, int64_t n_trees) {
    if (!g || n_trees < 0) return KC_ERR_INVALID_ARG;
    if (n_trees == 0) return KC_OK;
    try {
        clear_stale_error();
        ensure_pool(g, g->pool + n_trees);
        Plan p = plan_for(g, n_trees, false);
        ensure_ws(g, p);
        if (g->walker == KC_WALK_WARP) ensure_pipeline(g, p.BW);
        KC_CK(g, cudaStreamSynchronize(g->stream));
    } catch (Fail &f) {
        return f.st;
    }
    return KC_OK;
}

kc_status kc_sample_multi(kc_graph *const *graphs, const uint64_t *seeds, const int64_t *n_trees,
                          int32_t count) {
    if (!graphs || !seeds || !n_trees || count <= 0) return KC_ERR_INVALID_ARG;
    for (int32_t i = 0; i < count; ++i) {
        kc_graph *g = graphs[i];
        if (!g || n_trees[i] < 0) return KC_ERR_INVALID_ARG;
        for (int32_t j = 0; j < i; ++j)
            if (graphs[j] == g) return KC_ERR_INVALID_ARG;
        if (g->device != graphs[0]->device) return KC_ERR_INVALID_ARG;
        if (g->cfg.reject_steps > 0) return KC_ERR_INVALID_ARG;
        if (g->seeded && seeds[i] != g->seed) {
            g->last_error = "kc_sample_multi: the handle is already seeded with a different seed";
            return KC_ERR_INVALID_ARG;
        }
        if (g->next_sid + n_trees[i] > ((int64_t)1 << 32)) return KC_ERR_INVALID_ARG;
    }
    std::vector<char> was((size_t)count);
    for (int32_t i = 0; i < count; ++i) {
        was[(size_t)i] = graphs[i]->seeded;
        graphs[i]->seed = seeds[i];
        graphs[i]->seeded = true;
    }
    try {
        clear_stale_error();
        do_sample_multi(graphs, n_trees, count);
    } catch (Fail &f) {
        for (int32_t i = 0; i < count; ++i) graphs[i]->seeded = was[(size_t)i];
        return f.st;
    }
    return KC_OK;
}

kc_status kc_estimate(kc_graph *g, double eps, double delta, double *K_out) {
    if (!g || !K_out) return KC_ERR_INVALID_ARG;
    if (eps > 0 && !(delta > 0 && delta < 1)) return KC_ERR_INVALID_ARG;
    // an unseeded handle samples with seed 0; a call that adds no tree leaves
    // the handle unseeded
    const bool was_seeded = g->seeded;
    const int64_t pool0 = g->pool;
    try {
        clear_stale_error();
        if (eps > 0 && !g->seeded) {
            g->seed = 0;
            g->seeded = true;
        }
        const int64_t cap = g->cfg.max_trees > 0 ? g->cfg.max_trees : ((int64_t)1 << 24);
        const int64_t batch = g->cfg.batch_trees > 0 ? g->cfg.batch_trees : 1024;
        if (eps > 0) {
            if (g->cfg.stop_rule == KC_STOP_HOEFFDING) {
                const int64_t want = kc_host::hoeffding_trees(g->n, g->m, g->ecc, eps, delta, cap);
                if (want > g->pool) do_sample(g, want - g->pool);
            } else {
                kc_host::run_clt(
                    delta, eps, batch, cap, g->pool, [&](int64_t k) { do_sample(g, k); },
                    [&] {
                        const PoolSums s = reduce_pool(g);
                        return kc_host::Moments{s.count, s.wf, s.w, s.x2};
                    });
            }
        }
        if (g->pool == 0) {
            g->seeded = was_seeded;
            return KC_ERR_NO_SAMPLES;
        }
        PoolSums s = reduce_pool(g);
        bool unit = true;
        for (int64_t k = 0; k < g->pool && unit; ++k) unit = !g->h_modified[(size_t)k];
        if (unit && s.w == (double)s.count) {
            *K_out = i128_to_double(s.f_hi, s.f_lo) / ((double)(2 * g->m) * (double)s.count);
        } else {
            *K_out = s.wf / s.w;
        }
    } catch (Fail &f) {
        if (g->pool == pool0) g->seeded = was_seeded;
        return f.st;
    }
    return KC_OK;
}

kc_status kc_get_samples(kc_graph *g, int64_t first, int64_t count, int64_t *f, double *weight,
                         int64_t *steps, int64_t *sample_id) {
    if (!g || first < 0 || count < 0 || first + count > g->pool) return KC_ERR_INVALID_ARG;
    if (count == 0) return KC_OK;
    try {
        clear_stale_error();
        if (f) KC_CK(g, cudaMemcpyAsync(f, g->d_f + first, sizeof(int64_t) * count, cudaMemcpyDeviceToHost, g->stream));
        if (weight) KC_CK(g, cudaMemcpyAsync(weight, g->d_w + first, sizeof(double) * count, cudaMemcpyDeviceToHost, g->stream));
        if (steps) KC_CK(g, cudaMemcpyAsync(steps, g->d_steps + first, sizeof(int64_t) * count, cudaMemcpyDeviceToHost, g->stream));
        if (sample_id) KC_CK(g, cudaMemcpyAsync(sample_id, g->d_sid + first, sizeof(int64_t) * count, cudaMemcpyDeviceToHost, g->stream));
        KC_CK(g, cudaStreamSynchronize(g->stream));
    } catch (Fail &e) {
        return e.st;
    }
    return KC_OK;
}

kc_status kc_get_tau0(kc_graph *g, int32_t *p0, int32_t *level, int32_t *in0, int32_t *out0,
                      int32_t *root, int32_t *ecc) {
    if (!g) return KC_ERR_INVALID_ARG;
    try {
        clear_stale_error();
        const size_t b = sizeof(int32_t) * (size_t)g->n;
        if (p0) KC_CK(g, cudaMemcpyAsync(p0, g->d_p0, b, cudaMemcpyDeviceToHost, g->stream));
        if (level) KC_CK(g, cudaMemcpyAsync(level, g->d_level0, b, cudaMemcpyDeviceToHost, g->stream));
        if (in0) KC_CK(g, cudaMemcpyAsync(in0, g->d_in0, b, cudaMemcpyDeviceToHost, g->stream));
        if (out0) KC_CK(g, cudaMemcpyAsync(out0, g->d_out0, b, cudaMemcpyDeviceToHost, g->stream));
        KC_CK(g, cudaStreamSynchronize(g->stream));
        if (root) *root = g->root;
        if (ecc) *ecc = g->ecc;
    } catch (Fail &e) {
        return e.st;
    }
    return KC_OK;
}

kc_status kc_get_tree(kc_graph *g, int64_t sample, int32_t *parent, int32_t *depth,
                      int32_t *dfn_in, int32_t *dfn_out, int64_t *vol, int64_t *f,
                      int64_t *steps) {
    if (!g || sample < 0 || sample >= g->pool) return KC_ERR_INVALID_ARG;
    if (g->h_modified[(size_t)sample] && !g->cfg.keep_trees) return KC_ERR_NOT_RETAINED;
    if (g->cfg.keep_trees) {
        // retained tree (possibly drawn on an earlier version of the graph or
        // changed by an update): traverse its stored parent array on the
        // current graph; f and the step count are the pool's
        try {
        clear_stale_error();
            const int64_t n = g->n;
            GraphView gv = view_of(g);
            Plan p;
            p.BW = 1;
            p.BT = 1;
            p.bit = g->ttf_variant == KC_TTF_BIT;
            ensure_ws(g, p);
            UpdBuf ub = upd_buf(g);
            KC_CK(g, cudaMemcpyAsync(ub.slots, &sample, sizeof(int64_t), cudaMemcpyHostToDevice,
                                     g->stream));
            KC_CK(g, cudaMemsetAsync(g->d_err, 0, 2 * sizeof(uint32_t), g->stream));
            Carved c = carve(g, p);
            WaveView w = c.wv;
            w.B = 1;
            KC_CK(g, launch_prepare_from_parents(n, 1, g->root, g->d_parents, ub.slots, w,
                                                 g->stream));
            uint32_t hdr[2] = {0, 0};
            KC_CK(g, cudaMemcpyAsync(hdr, g->d_err, sizeof(hdr), cudaMemcpyDeviceToHost, g->stream));
            KC_CK(g, cudaStreamSynchronize(g->stream));
            if (hdr[0]) check_err(g, "get_tree");
            if (p.bit) {
                ensure_stack(g, p, hdr[1]);
                c = carve(g, p);
                w = c.wv;
                w.B = 1;
            }
            int nl = 0;
            KC_CK(g, launch_traverse(gv, w, p.bit, g->stream, &nl));
            if (p.bit) KC_CK(g, launch_ttf_bit(gv, w, g->stream));
            else KC_CK(g, launch_ttf_scan(gv, w, g->stream));
            check_err(g, "get_tree");
            std::vector<uint64_t> word((size_t)n);
            std::vector<int32_t> din((size_t)n), size((size_t)n);
            KC_CK(g, copy_sync(g, word.data(), w.word, sizeof(uint64_t) * n, cudaMemcpyDeviceToHost));
            KC_CK(g, copy_sync(g, din.data(), w.din, sizeof(int32_t) * n, cudaMemcpyDeviceToHost));
            KC_CK(g, copy_sync(g, size.data(), w.size, sizeof(int32_t) * n, cudaMemcpyDeviceToHost));
            if (vol) KC_CK(g, copy_sync(g, vol, w.vol, sizeof(int64_t) * n, cudaMemcpyDeviceToHost));
            if (f) KC_CK(g, copy_sync(g, f, g->d_f + sample, sizeof(int64_t), cudaMemcpyDeviceToHost));
            if (steps) KC_CK(g, copy_sync(g, steps, g->d_steps + sample, sizeof(int64_t),
                                           cudaMemcpyDeviceToHost));
            for (int64_t v = 0; v < n; ++v) {
                if (parent) parent[v] = w_next(word[(size_t)v]);
                if (depth) depth[v] = (int32_t)w_count(word[(size_t)v]);
                if (dfn_in) dfn_in[v] = din[(size_t)v];
                if (dfn_out) dfn_out[v] = din[(size_t)v] + size[(size_t)v] - 1;
            }
        } catch (Fail &e) {
            return e.st;
        }
        return KC_OK;
    }
    try {
        int64_t sid = 0;
        KC_CK(g, copy_sync(g, &sid, g->d_sid + sample, sizeof(int64_t), cudaMemcpyDeviceToHost));
        Plan p;
        p.BW = 1;
        p.BT = 1;
        p.bit = g->ttf_variant == KC_TTF_BIT;
        p.stack_cap = p.bit ? 4096 : 0;
        ensure_ws(g, p);
        run_wave(g, p, 1, sid, true);
        Carved c = carve(g, p);
        const int64_t n = g->n;
        std::vector<uint64_t> word((size_t)n);
        std::vector<int32_t> din((size_t)n), size((size_t)n);
        KC_CK(g, copy_sync(g, word.data(), c.wv.word, sizeof(uint64_t) * n, cudaMemcpyDeviceToHost));
        KC_CK(g, copy_sync(g, din.data(), c.wv.din, sizeof(int32_t) * n, cudaMemcpyDeviceToHost));
        KC_CK(g, copy_sync(g, size.data(), c.wv.size, sizeof(int32_t) * n, cudaMemcpyDeviceToHost));
        if (vol) KC_CK(g, copy_sync(g, vol, c.wv.vol, sizeof(int64_t) * n, cudaMemcpyDeviceToHost));
        if (f) KC_CK(g, copy_sync(g, f, c.wv.f, sizeof(int64_t), cudaMemcpyDeviceToHost));
        if (steps) KC_CK(g, copy_sync(g, steps, c.wv.steps, sizeof(int64_t), cudaMemcpyDeviceToHost));
        for (int64_t v = 0; v < n; ++v) {
            if (parent) parent[v] = w_next(word[(size_t)v]);
            if (depth) depth[v] = (int32_t)w_count(word[(size_t)v]);
            if (dfn_in) dfn_in[v] = din[(size_t)v];
            if (dfn_out) dfn_out[v] = din[(size_t)v] + size[(size_t)v] - 1;
        }
    } catch (Fail &e) {
        return e.st;
    }
    return KC_OK;
}

kc_status kc_stats(kc_graph *g, kc_stats_t *out) {
    if (!g || !out) return KC_ERR_INVALID_ARG;
    std::memset(out, 0, sizeof(*out));
    out->n = g->n;
    out->m = g->m;
    out->root = g->root;
    out->ecc = g->ecc;
    out->ttf_variant = g->ttf_variant;
    out->walker = g->walker;
    out->pool_trees = g->pool;
    out->next_sample_id = g->next_sid;
    out->trees_in_flight = g->last_wave;
    out->pool_bytes = g->pool_cap * (int64_t)(8 + 8 + 8 + 8) +
                      (g->cfg.keep_trees ? g->pool_cap * g->n * 4 : 0);
    out->workspace_bytes = (int64_t)(g->ws_bytes + g->stack_bytes);
    out->updates_applied = g->updates_applied;
    out->trees_resampled = g->trees_resampled;
    out->last_resistance = g->last_r;
    out->last_cg_iters = g->last_cg_iters;
    out->traversal = fast_traversal(g) == kTravLeafUp ? 2 : 1;
    out->tuned = g->tuned ? 1 : 0;
    for (int k = 0; k < 4; ++k) out->tune_ms[k] = g->tune_ms[k];
    out->resident_trees = g->resident_trees;
    out->trees_rejected = g->trees_rejected;
    out->ms_wilson = g->t_wilson.ms;
    out->ms_traverse = g->t_traverse.ms;
    out->ms_ttf = g->t_ttf.ms;
    out->ms_reduce = g->t_reduce.ms;
    out->ms_update = g->t_update.ms;
    out->ms_setup = g->t_setup.ms;
    out->ms_wave_init = g->t_init.ms;
    out->launches_wave_init = g->t_init.launches;
    out->launches_wilson = g->t_wilson.launches;
    out->launches_traverse = g->t_traverse.launches;
    out->launches_ttf = g->t_ttf.launches;
    out->launches_reduce = g->t_reduce.launches;
    out->launches_update = g->t_update.launches;
    out->launches_setup = g->t_setup.launches;
    out->ms_update_graph = g->ms_upd_part[0];
    out->ms_update_resistance = g->ms_upd_part[1];
    out->ms_update_trees = g->ms_upd_part[2] - g->ms_upd_part[3];  // refreshes timed apart
    out->ms_update_refresh = g->ms_upd_part[3];
    if (g->pool > 0) {
        try {
            std::vector<int64_t> st((size_t)g->pool);
            KC_CK(g, copy_sync(g, st.data(), g->d_steps, sizeof(int64_t) * g->pool,
                                cudaMemcpyDeviceToHost));
            int64_t tot = 0;
            for (int64_t x : st) tot += x;
            out->total_steps = tot;
            PoolSums s{};
            KC_CK(g, launch_pool_reduce(g->d_f, g->d_w, g->pool, 2 * g->m, g->d_scratch, g->stream));
            KC_CK(g, copy_sync(g, &s, g->d_scratch, sizeof(s), cudaMemcpyDeviceToHost));
            out->f_sum_hi = s.f_hi;
            out->f_sum_lo = s.f_lo;
            out->wf_sum = s.wf;
            out->w_sum = s.w;
            out->x2_sum = s.x2;
        } catch (Fail &e) {
            return e.st;
        }
    }
    return KC_OK;
}

kc_status kc_get_pool_sums(kc_graph *g, kc_pool_sums *out) {
    if (!g || !out) return KC_ERR_INVALID_ARG;
    std::memset(out, 0, sizeof(*out));
    if (g->pool == 0) return KC_OK;
    try {
        clear_stale_error();
        const PoolSums s = reduce_pool(g);
        out->f_sum_hi = s.f_hi;
        out->f_sum_lo = s.f_lo;
        out->wf_sum = s.wf;
        out->w_sum = s.w;
        out->x2_sum = s.x2;
        out->count = s.count;
    } catch (Fail &f) {
        return f.st;
    }
    return KC_OK;
}

kc_status kc_combine_sums(const kc_pool_sums *parts, int32_t count, kc_pool_sums *out) {
    if (!parts || !out || count < 1) return KC_ERR_INVALID_ARG;
    __int128 f = 0;
    kc_pool_sums r{};
    for (int32_t i = 0; i < count; ++i) {
        const kc_pool_sums &p = parts[i];
        const __int128 v = ((__int128)p.f_sum_hi << 64) | (__int128)p.f_sum_lo;
        if (__builtin_add_overflow(f, v, &f)) return KC_ERR_INVALID_ARG;
        r.wf_sum += p.wf_sum;
        r.w_sum += p.w_sum;
        r.x2_sum += p.x2_sum;
        if (p.count < 0 || __builtin_add_overflow(r.count, p.count, &r.count))
            return KC_ERR_INVALID_ARG;
    }
    r.f_sum_hi = (int64_t)(f >> 64);
    r.f_sum_lo = (uint64_t)f;
    *out = r;
    return KC_OK;
}

kc_status kc_estimate_from_sums(const kc_pool_sums *s, int64_t twom, int32_t unit_weights,
                                double *K_out) {
    if (!s || !K_out || twom < 2 || s->count < 1) return KC_ERR_INVALID_ARG;
    if (unit_weights) {
        *K_out = i128_to_double(s->f_sum_hi, s->f_sum_lo) / ((double)twom * (double)s->count);
        return KC_OK;
    }
    if (!(s->w_sum > 0)) return KC_ERR_INVALID_ARG;
    *K_out = s->wf_sum / s->w_sum;
    return KC_OK;
}

kc_status kc_reset_timers(kc_graph *g) {
    if (!g) return KC_ERR_INVALID_ARG;
    g->t_wilson = g->t_traverse = g->t_ttf = g->t_reduce = g->t_update = g->t_setup =
        g->t_init = PhaseTimer();
    for (double &x : g->ms_upd_part) x = 0.0;
    return KC_OK;
}

kc_status kc_update(kc_graph *g, const kc_edge_op *ops, int64_t n_ops, int32_t mode) {
    if (!g || (n_ops > 0 && !ops) || n_ops < 0) return KC_ERR_INVALID_ARG;
    if (mode != KC_UPDATE_BSM && mode != KC_UPDATE_ISM) return KC_ERR_INVALID_ARG;
    if (g->cfg.tau0_kind != KC_TAU0_BFS) {
        g->last_error = "kc_update: sample maintenance rebuilds tau0 as a BFS tree; "
                        "create the handle with tau0_kind = KC_TAU0_BFS";
        return KC_ERR_INVALID_ARG;
    }
    if (!g->cfg.keep_trees) return KC_ERR_NOT_RETAINED;
    if (g->pool == 0) return KC_ERR_NO_SAMPLES;
    if (n_ops == 0) return KC_OK;
    try {
        clear_stale_error();
        const kc_status st = validate_batch(g, ops, n_ops);
        if (st != KC_OK) return st;
        KC_CK(g, cudaEventRecord(g->ev0, g->stream));
        for (int64_t i = 0; i < n_ops; ++i) {
            const kc_edge_op &o = ops[i];
            if (o.op == 0) apply_insert(g, o.u, o.v, mode, o.r);
            else apply_delete(g, o.u, o.v, mode);
            ++g->updates_applied;
            ++g->update_seq;
        }
        KC_CK(g, cudaEventRecord(g->ev1, g->stream));
        KC_CK(g, cudaEventSynchronize(g->ev1));
        float ms = 0.f;
        KC_CK(g, cudaEventElapsedTime(&ms, g->ev0, g->ev1));
        g->t_update.ms += ms;
        sync_host_csr(g);
    } catch (Fail &f) {
        // ops applied before the failure stay applied: keep the host copy in step
        try {
            sync_host_csr(g);
        } catch (Fail &) {
        }
        return f.st;
    }
    return KC_OK;
}

}  // extern "C"
