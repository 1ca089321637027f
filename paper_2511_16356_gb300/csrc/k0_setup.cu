// Graph setup on the device: CSR validation, walk records, root choice, the
// BFS tree tau0 (Algorithm 1, "Generate tau0 using BFS with root r") and a
// parent-first order of tau0 for the traversal passes.
#include "kc_common.cuh"

namespace kc {

namespace {

__global__ void k_build_records(GraphView g, VRec *rec, int32_t *deg) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= g.n) return;
    const int64_t off = g.row_off[v];
    const int32_t d = (int32_t)(g.row_off[v + 1] - off);
    VRec r;
    r.deg = d;
    r.off_lo = (uint32_t)off;
    r.off_hi = (uint32_t)((uint64_t)off >> 32);
#pragma unroll
    for (int k = 0; k < kInline; ++k) r.nbr[k] = k < d ? g.col[off + k] : -1;
    rec[v] = r;
    deg[v] = d;
}

// flags: 1 column out of range, 2 self loop, 4 row not strictly ascending,
//        8 missing reverse edge, 16 isolated vertex
__global__ void k_validate(GraphView g, uint32_t *flags) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t n = g.n;
    if (e < n && g.row_off[e + 1] == g.row_off[e]) atomicOr(flags, 16u);
    if (e >= g.twom) return;
    // source row of entry e: largest v with row_off[v] <= e
    int64_t lo = 0, hi = n - 1;
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (g.row_off[mid] <= e) lo = mid; else hi = mid - 1;
    }
    const int64_t v = lo;
    const int32_t w = g.col[e];
    uint32_t f = 0;
    if (w < 0 || w >= n) { atomicOr(flags, 1u); return; }
    if (w == v) f |= 2u;
    if (e + 1 < g.row_off[v + 1] && g.col[e + 1] <= w) f |= 4u;
    // reverse edge (w, v) by binary search in row w
    int64_t a = g.row_off[w], b = g.row_off[w + 1] - 1;
    bool found = false;
    while (a <= b) {
        const int64_t mid = (a + b) >> 1;
        const int32_t c = g.col[mid];
        if (c == v) { found = true; break; }
        if (c < v) a = mid + 1; else b = mid - 1;
    }
    if (!found) f |= 8u;
    if (f) atomicOr(flags, f);
}

// Highest degree, smallest id on ties: maximise (deg << 32) | (2^32 - 1 - v).
__global__ void k_root(GraphView g, unsigned long long *best) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= g.n) return;
    const unsigned long long key =
        ((unsigned long long)(uint32_t)g.deg[v] << 32) | (0xFFFFFFFFull - (unsigned long long)v);
    atomicMax(best, key);
}

__global__ void k_bfs_init(int64_t n, int32_t r, int32_t *level) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n) level[v] = (v == r) ? 0 : -1;
}

// One level-synchronous BFS round: every vertex on level `lev` labels its
// unlabelled neighbours lev + 1 (all writers store the same value).
__global__ void k_bfs_level(GraphView g, int32_t lev, int32_t *level, int32_t *changed) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= g.n || level[v] != lev) return;
    bool any = false;
    for (int64_t e = g.row_off[v]; e < g.row_off[v + 1]; ++e) {
        const int32_t w = g.col[e];
        if (level[w] < 0) { level[w] = lev + 1; any = true; }
    }
    if (any) *changed = 1;
}

// tau0 parent: the smallest-id neighbour one level closer to r (rows ascend).
__global__ void k_bfs_parent(GraphView g, const int32_t *level, int32_t *p0, int32_t *unreached) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= g.n) return;
    const int32_t lv = level[v];
    if (lv < 0) { atomicAdd(unreached, 1); p0[v] = -1; return; }
    int32_t p = -1;
    if (lv > 0) {
        for (int64_t e = g.row_off[v]; e < g.row_off[v + 1]; ++e) {
            const int32_t w = g.col[e];
            if (level[w] == lv - 1) { p = w; break; }
        }
    }
    p0[v] = p;
}

__global__ void k_tau0_words(int64_t n, const int32_t *p0, const int32_t *level, uint64_t *word) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n) word[v] = w_make(p0[v], (uint32_t)level[v], true);
}

__global__ void k_level_hist(int64_t n, const int32_t *level, int32_t *hist) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n) atomicAdd(hist + level[v], 1);
}

// exclusive scan of hist[0..L] in place by one block (L is the eccentricity + 1)
__global__ void k_scan_small(int32_t *hist, int32_t L) {
    __shared__ int32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int32_t base = 0; base < L; base += blockDim.x) {
        const int32_t i = base + threadIdx.x;
        int32_t x = i < L ? hist[i] : 0;
        // block inclusive scan (Hillis-Steele in shared memory)
        __shared__ int32_t buf[1024];
        buf[threadIdx.x] = x;
        __syncthreads();
        for (int d = 1; d < (int)blockDim.x; d <<= 1) {
            const int32_t y = threadIdx.x >= (unsigned)d ? buf[threadIdx.x - d] : 0;
            __syncthreads();
            buf[threadIdx.x] += y;
            __syncthreads();
        }
        const int32_t incl = buf[threadIdx.x];
        const int32_t c = carry;
        if (i < L) hist[i] = c + incl - x;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = c + incl;
        __syncthreads();
    }
}

__global__ void k_level_scatter(int64_t n, const int32_t *level, int32_t *offs, int32_t *ord) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n) ord[atomicAdd(offs + level[v], 1)] = (int32_t)v;
}

// max over v of (score << 32 | (2^32 - 1 - v)): largest score, smallest id.
// mode 0: score = level a; mode 1: score = min(level a, level b)
__global__ void k_argmax_score(int64_t n, const int32_t *la, const int32_t *lb, int mode,
                               unsigned long long *best) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    const int32_t sc = mode == 0 ? la[v] : min(la[v], lb[v]);
    atomicMax(best, ((unsigned long long)(uint32_t)sc << 32) | (0xFFFFFFFFull - (unsigned long long)v));
}

// among vertices of degree dmax: min of (max(la, lb, lc) << 32 | v); also counts them
__global__ void k_central_pick(int64_t n, const int32_t *deg, int32_t dmax, const int32_t *la,
                               const int32_t *lb, const int32_t *lc, unsigned long long *best,
                               int32_t *ties) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n || deg[v] != dmax) return;
    atomicAdd(ties, 1);
    if (!la) return;
    const int32_t e = max(la[v], max(lb[v], lc[v]));
    atomicMin(best, ((unsigned long long)(uint32_t)e << 32) | (unsigned long long)v);
}

// Depth-first tree from r (rows in ascending id): one thread with an explicit
// stack of (vertex, next row position) -- the recursive DFS is inherently
// sequential.  Every iteration either advances a row position or pops, so the
// loop ends after at most 2m + n iterations.  level[] must be -1 everywhere.
__global__ void k_dfs_tree(GraphView g, int32_t r, int32_t *p0, int32_t *level, int32_t *sv,
                           int64_t *se, int32_t *deepest) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    const int64_t *__restrict__ row_off = g.row_off;
    const int32_t *__restrict__ col = g.col;
    int64_t sp = 0;
    int32_t dmax = 0;
    level[r] = 0;
    p0[r] = -1;
    sv[0] = r;
    se[0] = row_off[r];
    const int64_t cap = 2 * g.twom + 2 * g.n + 2;
    for (int64_t it = 0; sp >= 0 && it < cap; ++it) {
        const int32_t u = sv[sp];
        const int64_t e = se[sp];
        if (e < row_off[u + 1]) {
            const int32_t w = col[e];
            se[sp] = e + 1;
            if (level[w] < 0) {
                const int32_t lw = level[u] + 1;
                p0[w] = u;
                level[w] = lw;
                dmax = lw > dmax ? lw : dmax;
                ++sp;
                sv[sp] = w;
                se[sp] = row_off[w];
            }
        } else {
            --sp;
        }
    }
    *deepest = dmax;
}

__global__ void k_fill2(int64_t n, int32_t *a, int32_t *b, int32_t value) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n) {
        a[v] = value;
        b[v] = value;
    }
}

// tau0 from a sampled tree's walker words: parent and depth; counts vertices
// outside the tree and records the largest depth
__global__ void k_tau0_from_words(int64_t n, const uint64_t *word, int32_t *p0, int32_t *level,
                                  int32_t *deepest, int32_t *outside) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    const uint64_t x = word[v];
    if (!w_in_tree(x)) {
        atomicAdd(outside, 1);
        p0[v] = -1;
        level[v] = -1;
        return;
    }
    p0[v] = w_next(x);
    level[v] = (int32_t)w_count(x);
    atomicMax(deepest, (int32_t)w_count(x));
}

__global__ void k_count_negative(int64_t n, const int32_t *a, int32_t *count) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n && a[v] < 0) atomicAdd(count, 1);
}

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

cudaError_t launch_dfs_tree(const GraphView &g, int32_t r, int32_t *p0, int32_t *level,
                            int32_t *sv, int64_t *se, int32_t *deepest, int32_t *unreached,
                            cudaStream_t s) {
    k_fill2<<<blocks_for(g.n, 256), 256, 0, s>>>(g.n, p0, level, -1);
    k_dfs_tree<<<1, 1, 0, s>>>(g, r, p0, level, sv, se, deepest);
    k_count_negative<<<blocks_for(g.n, 256), 256, 0, s>>>(g.n, level, unreached);
    return cudaGetLastError();
}

cudaError_t launch_tau0_from_words(int64_t n, const uint64_t *word, int32_t *p0, int32_t *level,
                                   int32_t *deepest, int32_t *outside, cudaStream_t s) {
    k_tau0_from_words<<<blocks_for(n, 256), 256, 0, s>>>(n, word, p0, level, deepest, outside);
    return cudaGetLastError();
}

cudaError_t launch_argmax_score(int64_t n, const int32_t *la, const int32_t *lb, int mode,
                                unsigned long long *best, cudaStream_t s) {
    k_argmax_score<<<blocks_for(n, 256), 256, 0, s>>>(n, la, lb, mode, best);
    return cudaGetLastError();
}

cudaError_t launch_central_pick(int64_t n, const int32_t *deg, int32_t dmax, const int32_t *la,
                                const int32_t *lb, const int32_t *lc, unsigned long long *best,
                                int32_t *ties, cudaStream_t s) {
    k_central_pick<<<blocks_for(n, 256), 256, 0, s>>>(n, deg, dmax, la, lb, lc, best, ties);
    return cudaGetLastError();
}

cudaError_t launch_build_records(const GraphView &g, VRec *rec, int32_t *deg, cudaStream_t s) {
    k_build_records<<<blocks_for(g.n, 256), 256, 0, s>>>(g, rec, deg);
    return cudaGetLastError();
}

cudaError_t launch_validate(const GraphView &g, uint32_t *flags, cudaStream_t s) {
    const int64_t work = g.twom > g.n ? g.twom : g.n;
    k_validate<<<blocks_for(work, 256), 256, 0, s>>>(g, flags);
    return cudaGetLastError();
}

cudaError_t launch_root(const GraphView &g, unsigned long long *best, cudaStream_t s) {
    k_root<<<blocks_for(g.n, 256), 256, 0, s>>>(g, best);
    return cudaGetLastError();
}

cudaError_t launch_bfs_init(int64_t n, int32_t r, int32_t *level, cudaStream_t s) {
    k_bfs_init<<<blocks_for(n, 256), 256, 0, s>>>(n, r, level);
    return cudaGetLastError();
}

cudaError_t launch_bfs_level(const GraphView &g, int32_t lev, int32_t *level, int32_t *changed,
                             cudaStream_t s) {
    k_bfs_level<<<blocks_for(g.n, 256), 256, 0, s>>>(g, lev, level, changed);
    return cudaGetLastError();
}

cudaError_t launch_bfs_parent(const GraphView &g, const int32_t *level, int32_t *p0,
                              int32_t *unreached, cudaStream_t s) {
    k_bfs_parent<<<blocks_for(g.n, 256), 256, 0, s>>>(g, level, p0, unreached);
    return cudaGetLastError();
}

cudaError_t launch_tau0_words(int64_t n, const int32_t *p0, const int32_t *level, uint64_t *word,
                              cudaStream_t s) {
    k_tau0_words<<<blocks_for(n, 256), 256, 0, s>>>(n, p0, level, word);
    return cudaGetLastError();
}

// Parent-first order of tau0: vertices sorted by BFS level (order inside a
// level is irrelevant to the traversal passes).  hist needs ecc + 1 entries.
cudaError_t launch_level_order(int64_t n, int32_t ecc, const int32_t *level, int32_t *hist,
                               int32_t *ord, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(hist, 0, sizeof(int32_t) * (size_t)(ecc + 1), s);
    if (e != cudaSuccess) return e;
    k_level_hist<<<blocks_for(n, 256), 256, 0, s>>>(n, level, hist);
    k_scan_small<<<1, 1024, 0, s>>>(hist, ecc + 1);
    k_level_scatter<<<blocks_for(n, 256), 256, 0, s>>>(n, level, hist, ord);
    return cudaGetLastError();
}

}  // namespace kc
