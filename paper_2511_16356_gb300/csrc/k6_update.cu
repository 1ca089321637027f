// Sample maintenance kernels (Sec. 4): BSM (Algorithm 2) and ISM (Algorithm 3).
//
//  - conditioned Wilson: walker words initialised with the edge (u, v) already
//    in the tree (u -> v, root v); the result is re-rooted at r;
//  - containment scan of the pool for an edge, Floyd selection of the trees to
//    replace or transform (Philox select stream);
//  - preparation of retained trees for the traversal passes: children lists,
//    then a warp-per-tree breadth-first pass giving depths and a parent-first
//    order;
//  - link-cut (ISM insertion) and cut-link (ISM deletion), one warp per tree;
//  - weight rescaling with sums in a fixed order (bit-reproducible).
// The random choices follow the oracle's contract: tags select / link-cut /
// cut-link with counters (update seq, draw index or pool index, 0).
#include "kc_common.cuh"

namespace kc {

namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;

__global__ void k_edge_pre_init(int64_t n, int64_t B, int32_t u, int32_t v, uint64_t *word,
                                int32_t *ord) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= B) return;
    word[t * n + v] = w_make(-1, 0, true);
    word[t * n + u] = w_make(v, 1, true);
    ord[t * n] = v;
    ord[t * n + 1] = u;
}

// dst[slot[t]][x] = parent of x in wave tree t
__global__ void k_words_to_slots(int64_t n, int64_t B, const uint64_t *word, const int64_t *slot,
                                 int32_t *pool_parents) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= B * n) return;
    const int64_t t = k / n, x = k - t * n;
    pool_parents[slot[t] * n + x] = w_next(word[k]);
}

// reverse the parent chain from r up to the old root `top` in each slot tree
__global__ void k_reroot_slots(int64_t n, int64_t B, const int64_t *slot, int32_t *pool_parents,
                               int32_t r, int32_t top, uint32_t *err) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= B || r == top) return;
    int32_t *p = pool_parents + slot[t] * n;
    int32_t prev = -1, cur = r;
    for (int64_t it = 0; it <= n; ++it) {
        const int32_t nxt = p[cur];
        p[cur] = prev;
        if (cur == top) return;
        if (nxt < 0 || nxt >= n) break;
        prev = cur;
        cur = nxt;
    }
    atomicOr(err, kErrBadTree);
}

__global__ void k_contains_edge(int64_t n, int64_t P, const int32_t *pool_parents, int32_t u,
                                int32_t v, uint8_t *flag) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P) return;
    const int32_t *p = pool_parents + i * n;
    flag[i] = (p[u] == v || p[v] == u) ? 1 : 0;
}

// Floyd's sampling of k of [0, N) (one thread; `taken` zeroed, N bytes)
__global__ void k_select_floyd(uint64_t seed, uint32_t seq, int64_t N, int64_t k, uint8_t *taken,
                               int64_t *out) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    int64_t cnt = 0;
    for (int64_t j = N - k; j < N; ++j) {
        int64_t tt = (int64_t)bounded_draw(seed, seq, (uint32_t)cnt, 0, kTagSelect, (uint32_t)(j + 1));
        if (taken[tt]) tt = j;
        taken[tt] = 1;
        out[cnt++] = tt;
    }
}

// ---- preparation of parent arrays for the traversal passes ----------------
__global__ void k_gather_parents(int64_t n, int64_t B, const int32_t *pool_parents,
                                 const int64_t *slot, uint64_t *word, int32_t *cnt) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= B * n) return;
    const int64_t t = k / n;
    const int32_t p = pool_parents[slot[t] * n + (k - t * n)];
    word[k] = w_make(p, 0, false);
    if (p >= 0) atomicAdd(cnt + t * n + p, 1);
}

// exclusive scan of the child counts, warp per tree; off[t][n] is not stored
__global__ void __launch_bounds__(128) k_child_scan(int64_t n, int64_t B, const int32_t *cnt,
                                                    int32_t *off) {
    const int lane = threadIdx.x & 31;
    const int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (t >= B) return;
    int32_t carry = 0;
    for (int64_t base = 0; base < n; base += 32) {
        const int64_t x = base + lane;
        const int32_t c = x < n ? cnt[t * n + x] : 0;
        int32_t incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t y = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += y;
        }
        if (x < n) off[t * n + x] = carry + incl - c;
        carry += __shfl_sync(kFull, incl, 31);
    }
}

__global__ void k_child_scatter(int64_t n, int64_t B, const uint64_t *word, const int32_t *off,
                                int32_t *fill, int32_t *children) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= B * n) return;
    const int64_t t = k / n;
    const int32_t p = w_next(word[k]);
    if (p < 0) return;
    const int32_t pos = off[t * n + p] + atomicAdd(fill + t * n + p, 1);
    children[t * n + pos] = (int32_t)(k - t * n);
}

// Breadth-first order from the root (parent first) and depths, warp per tree.
__global__ void __launch_bounds__(128) k_bfs_order(int64_t n, int64_t B, int32_t root,
                                                   const int32_t *off, const int32_t *cnt,
                                                   const int32_t *children, uint64_t *word,
                                                   int32_t *ord, uint32_t *err,
                                                   int32_t *w_maxdepth) {
    const int lane = threadIdx.x & 31;
    const int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (t >= B) return;
    uint64_t *wd = word + t * n;
    int32_t *od = ord + t * n;
    const int32_t *ch = children + t * n;
    if (lane == 0) {
        od[0] = root;
        wd[root] = w_make(-1, 0, true);
    }
    __syncwarp();
    int64_t head = 0, tail = 1;
    while (head < tail) {
        const int64_t q = head + lane;
        int32_t v = -1, c = 0, o = 0;
        uint32_t dv = 0;
        if (q < tail) {  // entries written by other lanes: read at L2
            v = __ldcg(od + q);
            c = cnt[t * n + v];
            o = off[t * n + v];
            dv = w_count((uint64_t)__ldcg((const unsigned long long *)(wd + v)));
        }
        int32_t incl = c;
#pragma unroll
        for (int s = 1; s < 32; s <<= 1) {
            const int32_t y = __shfl_up_sync(kFull, incl, s);
            if (lane >= s) incl += y;
        }
        const int32_t total = __shfl_sync(kFull, incl, 31);
        int64_t pos = tail + incl - c;
        for (int32_t j = 0; j < c; ++j) {
            const int32_t x = ch[o + j];
            if (pos < n) {
                __stcg(od + pos, x);
                __stcg((unsigned long long *)(wd + x), (unsigned long long)w_make(v, dv + 1, true));
            }
            ++pos;
        }
        if (c > 0) atomicMax(w_maxdepth, (int)dv + 1);
        const int64_t took = min((int64_t)32, tail - head);
        head += took;
        tail += total;
        __threadfence_block();
        __syncwarp();
        if (tail > n) {
            if (lane == 0) atomicOr(err, kErrBadTree);
            return;
        }
    }
    if (tail != n && lane == 0) atomicOr(err, kErrBadTree);
}

// ---- link-cut / cut-link, one warp per selected tree -----------------------
struct TransformIn {
    int64_t n;
    const int64_t *row_off;   // G'
    const int32_t *col;
    const uint64_t *word;     // [B][n] parent + depth of the old tree
    const int32_t *din;       // [B][n] DFN of the old tree
    const int32_t *size;      // [B][n]
    const int32_t *pre;       // [B][n] preorder -> vertex
    int32_t *scratch;         // [B][>= n] int32 per tree (cut-link's per-position counts)
    const int64_t *slot;      // [B] pool index of each tree
    int32_t *pool_parents;    // [P][n] written in place
    double *factor;           // [B] d_old / d_new
    int32_t r, u, v;
    uint64_t seed;
    uint32_t seq;
    uint32_t *err;
};

__device__ int64_t tree_dist(const uint64_t *wd, int32_t a, int32_t b, int64_t n) {
    int64_t d = 0;
    int32_t da = (int32_t)w_count(wd[a]), db = (int32_t)w_count(wd[b]);
    for (int64_t it = 0; it < 2 * n + 2 && a != b; ++it) {
        if (da >= db) { a = w_next(wd[a]); --da; } else { b = w_next(wd[b]); --db; }
        ++d;
    }
    return d;
}

__device__ void reroot_chain(int32_t *p, int32_t x, int32_t top, int32_t attach, int64_t n,
                             uint32_t *err) {
    int32_t prev = attach, cur = x;
    for (int64_t it = 0; it <= n; ++it) {
        const int32_t nxt = p[cur];
        p[cur] = prev;
        if (cur == top) return;
        if (nxt < 0 || nxt >= n) break;
        prev = cur;
        cur = nxt;
    }
    atomicOr(err, kErrBadTree);
}

__global__ void __launch_bounds__(128) k_link_cut(TransformIn a, int64_t B) {
    const int lane = threadIdx.x & 31;
    const int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (t >= B) return;
    const int64_t n = a.n;
    const uint64_t *wd = a.word + t * n;
    const int32_t *din = a.din + t * n;
    const int32_t *sz = a.size + t * n;
    const int32_t *pre = a.pre + t * n;
    // path u..v: climb to the lowest common ancestor
    int32_t x = -1, side = -1;
    int64_t d_old = 0;
    if (lane == 0) {
        int32_t p = a.u, q = a.v;
        int32_t dp = (int32_t)w_count(wd[p]), dq = (int32_t)w_count(wd[q]);
        while (dp > dq) { p = w_next(wd[p]); --dp; }
        while (dq > dp) { q = w_next(wd[q]); --dq; }
        while (p != q) { p = w_next(wd[p]); q = w_next(wd[q]); }
        const int64_t du = (int64_t)w_count(wd[a.u]) - w_count(wd[p]);
        const int64_t dvv = (int64_t)w_count(wd[a.v]) - w_count(wd[p]);
        d_old = du + dvv;
        const int64_t k = (int64_t)bounded_draw(a.seed, a.seq, (uint32_t)a.slot[t], 0, kTagLinkCut,
                                                (uint32_t)d_old);
        if (k < du) {
            x = a.u;
            for (int64_t i = 0; i < k; ++i) x = w_next(wd[x]);
            side = a.u;
        } else {
            x = a.v;
            for (int64_t i = 0; i < k - du; ++i) x = w_next(wd[x]);
            side = a.v;
        }
        reroot_chain(a.pool_parents + a.slot[t] * n, side, x, side == a.u ? a.v : a.u, n, a.err);
    }
    x = __shfl_sync(kFull, x, 0);
    // edges of G' other than e that cross Sub(tau, x): an edge crosses the cut
    // from either side, so the scan runs over the smaller side (the preorder
    // positions of Sub(tau, x), or all the others)
    const int32_t lo = din[x], hi = din[x] + sz[x] - 1;
    const bool inside = 2 * (int64_t)sz[x] <= n;
    const int64_t span = inside ? (int64_t)sz[x] : n - sz[x];
    long long cross = 0;
    for (int64_t k = lane; k < span; k += 32) {
        const int64_t q = inside ? lo + k : (k < lo ? k : k + sz[x]);
        const int32_t y = pre[q];
        for (int64_t e = a.row_off[y]; e < a.row_off[y + 1]; ++e) {
            const int32_t z = a.col[e];
            const int32_t dz = din[z];
            if ((dz >= lo && dz <= hi) == inside) continue;  // both ends on the scanned side
            if ((y == a.u && z == a.v) || (y == a.v && z == a.u)) continue;
            ++cross;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cross += __shfl_down_sync(kFull, cross, o);
    if (lane == 0) a.factor[t] = cross > 0 ? (double)d_old / (double)cross : 0.0;
}

__global__ void __launch_bounds__(128) k_cut_link(TransformIn a, int64_t B) {
    const int lane = threadIdx.x & 31;
    const int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (t >= B) return;
    const int64_t n = a.n;
    const uint64_t *wd = a.word + t * n;
    const int32_t *din = a.din + t * n;
    const int32_t *sz = a.size + t * n;
    const int32_t *pre = a.pre + t * n;
    const int32_t c = (w_next(wd[a.u]) == a.v) ? a.u : a.v;
    const int32_t qv = (c == a.u) ? a.v : a.u;
    const int32_t lo = din[c], hi = din[c] + sz[c] - 1;
    // count crossing edges (G' no longer has e) from the smaller side of the
    // cut: the preorder positions of Sub(tau, c), or all the others
    const bool inside = 2 * (int64_t)sz[c] <= n;
    const int64_t span = inside ? (int64_t)sz[c] : n - sz[c];
    long long cross = 0;
    for (int64_t kq = lane; kq < span; kq += 32) {
        const int64_t q = inside ? lo + kq : (kq < lo ? kq : kq + sz[c]);
        const int32_t y = pre[q];
        for (int64_t e = a.row_off[y]; e < a.row_off[y + 1]; ++e) {
            const int32_t dz = din[a.col[e]];
            if ((dz >= lo && dz <= hi) != inside) ++cross;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cross += __shfl_xor_sync(kFull, cross, o);
    if (cross <= 0) {
        if (lane == 0) atomicOr(a.err, kErrBadTree);
        return;
    }
    long long k = 0;
    if (lane == 0)
        k = (long long)bounded_draw(a.seed, a.seq, (uint32_t)a.slot[t], 0, kTagCutLink,
                                    (uint32_t)cross);
    k = __shfl_sync(kFull, k, 0);
    // find the k-th crossing edge in (preorder position of the inside end,
    // outside end ascending) order
    int32_t ia = -1, ob = -1;
    long long before = 0;
    if (!inside) {
        // the outside is smaller: tally each inside position's crossing edges
        // from the outside (atomics in L2), then scan the tallies in order
        int32_t *cnt = a.scratch + t * n;
        for (int64_t i = lane; i < sz[c]; i += 32) __stcg(cnt + i, 0);
        __threadfence_block();
        __syncwarp();
        for (int64_t kq = lane; kq < span; kq += 32) {
            const int64_t q = kq < lo ? kq : kq + sz[c];
            const int32_t y = pre[q];
            for (int64_t e = a.row_off[y]; e < a.row_off[y + 1]; ++e) {
                const int32_t dz = din[a.col[e]];
                if (dz >= lo && dz <= hi) atomicAdd(cnt + (dz - lo), 1);
            }
        }
        __threadfence_block();
        __syncwarp();
        int64_t hit = -1;  // inside position (from lo) holding the k-th edge
        long long hit_start = 0;
        for (int64_t base = 0; base < sz[c] && hit < 0; base += 32) {
            const int64_t i = base + lane;
            const long long mine = i < sz[c] ? (long long)__ldcg(cnt + i) : 0;
            long long incl = mine;
#pragma unroll
            for (int s2 = 1; s2 < 32; s2 <<= 1) {
                const long long yv = __shfl_up_sync(kFull, incl, s2);
                if (lane >= s2) incl += yv;
            }
            const long long start = before + incl - mine;
            const unsigned hb = __ballot_sync(kFull, mine > 0 && k >= start && k < start + mine);
            if (hb) {
                const int src = __ffs(hb) - 1;
                hit = base + src;
                hit_start = __shfl_sync(kFull, start, src);
            }
            before += __shfl_sync(kFull, incl, 31);
        }
        if (lane == 0 && hit >= 0) {
            const int32_t y = pre[lo + hit];
            long long idx = hit_start;
            for (int64_t e = a.row_off[y]; e < a.row_off[y + 1]; ++e) {
                const int32_t z = a.col[e];
                const int32_t dz = din[z];
                if (dz >= lo && dz <= hi) continue;
                if (idx == k) { ia = y; ob = z; break; }
                ++idx;
            }
        }
    }
    for (int64_t base = lo; inside && base <= hi; base += 32) {
        const int64_t q = base + lane;
        int32_t y = -1;
        long long mine = 0;
        if (q <= hi) {
            y = pre[q];
            for (int64_t e = a.row_off[y]; e < a.row_off[y + 1]; ++e) {
                const int32_t dz = din[a.col[e]];
                if (dz < lo || dz > hi) ++mine;
            }
        }
        long long incl = mine;
#pragma unroll
        for (int s = 1; s < 32; s <<= 1) {
            const long long yv = __shfl_up_sync(kFull, incl, s);
            if (lane >= s) incl += yv;
        }
        const long long total = __shfl_sync(kFull, incl, 31);
        const long long start = before + incl - mine;
        const bool here = mine > 0 && k >= start && k < start + mine;
        const unsigned hb = __ballot_sync(kFull, here);
        if (hb) {
            if (here) {
                long long idx = start;
                for (int64_t e = a.row_off[y]; e < a.row_off[y + 1]; ++e) {
                    const int32_t z = a.col[e];
                    const int32_t dz = din[z];
                    if (dz >= lo && dz <= hi) continue;
                    if (idx == k) { ia = y; ob = z; break; }
                    ++idx;
                }
            }
            const int src = __ffs(hb) - 1;
            ia = __shfl_sync(kFull, ia, src);
            ob = __shfl_sync(kFull, ob, src);
            break;
        }
        before += total;
    }
    if (lane == 0) {
        if (ia < 0) {
            atomicOr(a.err, kErrBadTree);
            return;
        }
        const int64_t d_new = ((int64_t)w_count(wd[ia]) - w_count(wd[c])) + 1 +
                              tree_dist(wd, ob, qv, n);
        reroot_chain(a.pool_parents + a.slot[t] * n, ia, c, ob, n, a.err);
        a.factor[t] = (double)cross / (double)d_new;
    }
}

// ---- weights ----------------------------------------------------------------
// w[slot[j]] *= factor[j]
__global__ void k_scale_slots(double *w, const int64_t *slot, const double *factor, int64_t B) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < B) w[slot[j]] *= factor[j];
}

// sums over the pool in a fixed order: s[0] = sum over flagged, s[1] = unflagged
__global__ void __launch_bounds__(1024) k_weight_sums(const double *w, const uint8_t *flag,
                                                      int64_t P, double *s) {
    __shared__ double a[1024], b[1024];
    const int tid = threadIdx.x;
    double x = 0.0, y = 0.0;
    for (int64_t i = tid; i < P; i += blockDim.x) {
        if (flag[i]) x += w[i]; else y += w[i];
    }
    a[tid] = x;
    b[tid] = y;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if (tid < h) {
            a[tid] += a[tid + h];
            b[tid] += b[tid + h];
        }
        __syncthreads();
    }
    if (tid == 0) {
        s[0] = a[0];
        s[1] = b[0];
    }
}

// flagged weights -> w / A * target_flagged, unflagged -> w / B * target_rest
// (a target < 0 leaves that group unchanged)
__global__ void k_weight_rescale(double *w, const uint8_t *flag, int64_t P, const double *s,
                                 double target_flagged, double target_rest) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P) return;
    if (flag[i]) {
        if (target_flagged >= 0 && s[0] > 0) w[i] = w[i] / s[0] * target_flagged;
    } else {
        if (target_rest >= 0 && s[1] > 0) w[i] = w[i] / s[1] * target_rest;
    }
}

__global__ void k_scatter_results(const int64_t *slot, int64_t B, const int64_t *f,
                                  const int64_t *steps, const int64_t *sids, int64_t *pool_f,
                                  int64_t *pool_steps, int64_t *pool_sid) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= B) return;
    if (f) pool_f[slot[j]] = f[j];
    if (steps) pool_steps[slot[j]] = steps[j];
    if (sids) pool_sid[slot[j]] = sids[j];
}

inline unsigned blk(int64_t x, int t) { return (unsigned)((x + t - 1) / t); }

}  // namespace

cudaError_t launch_edge_pre_init(int64_t n, int64_t B, int32_t u, int32_t v, uint64_t *word,
                                 int32_t *ord, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(word, 0, sizeof(uint64_t) * (size_t)(B * n), s);
    if (e != cudaSuccess) return e;
    k_edge_pre_init<<<blk(B, 128), 128, 0, s>>>(n, B, u, v, word, ord);
    return cudaGetLastError();
}

cudaError_t launch_words_to_slots(int64_t n, int64_t B, const uint64_t *word, const int64_t *slot,
                                  int32_t *pool_parents, int32_t r, int32_t top, uint32_t *err,
                                  cudaStream_t s) {
    k_words_to_slots<<<blk(B * n, 256), 256, 0, s>>>(n, B, word, slot, pool_parents);
    if (top >= 0) k_reroot_slots<<<blk(B, 128), 128, 0, s>>>(n, B, slot, pool_parents, r, top, err);
    return cudaGetLastError();
}

cudaError_t launch_contains_edge(int64_t n, int64_t P, const int32_t *pool_parents, int32_t u,
                                 int32_t v, uint8_t *flag, cudaStream_t s) {
    k_contains_edge<<<blk(P, 256), 256, 0, s>>>(n, P, pool_parents, u, v, flag);
    return cudaGetLastError();
}

cudaError_t launch_select(uint64_t seed, uint32_t seq, int64_t N, int64_t k, uint8_t *taken,
                          int64_t *out, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(taken, 0, (size_t)N, s);
    if (e != cudaSuccess) return e;
    k_select_floyd<<<1, 1, 0, s>>>(seed, seq, N, k, taken, out);
    return cudaGetLastError();
}

// word/ord of wave trees from retained parent arrays: uses `cnt` (= size),
// `off` (= aux), `fill` (= din) and `children` (= vol reinterpreted) as scratch.
cudaError_t launch_prepare_from_parents(int64_t n, int64_t B, int32_t root,
                                        const int32_t *pool_parents, const int64_t *slot,
                                        WaveView w, cudaStream_t s) {
    const size_t per = sizeof(int32_t) * (size_t)(B * n);
    int32_t *cnt = w.size, *off = w.aux, *fill = w.din;
    int32_t *children = reinterpret_cast<int32_t *>(w.vol);
    cudaError_t e;
    if ((e = cudaMemsetAsync(cnt, 0, per, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(fill, 0, per, s)) != cudaSuccess) return e;
    k_gather_parents<<<blk(B * n, 256), 256, 0, s>>>(n, B, pool_parents, slot, w.word, cnt);
    k_child_scan<<<blk(B * 32, 128), 128, 0, s>>>(n, B, cnt, off);
    k_child_scatter<<<blk(B * n, 256), 256, 0, s>>>(n, B, w.word, off, fill, children);
    k_bfs_order<<<blk(B * 32, 128), 128, 0, s>>>(n, B, root, off, cnt, children, w.word, w.ord,
                                                 w.err, w.maxdepth);
    return cudaGetLastError();
}

cudaError_t launch_link_cut(const int64_t *row_off, const int32_t *col, WaveView w,
                            const int64_t *slot, int32_t *pool_parents, double *factor, int32_t r,
                            int32_t u, int32_t v, uint64_t seed, uint32_t seq, bool insert,
                            cudaStream_t s) {
    TransformIn a;
    a.n = w.n;
    a.row_off = row_off;
    a.col = col;
    a.word = w.word;
    a.din = w.din;
    a.size = w.size;
    a.pre = w.aux;
    a.scratch = reinterpret_cast<int32_t *>(w.vol);  // 8n bytes per tree, unused here
    a.slot = slot;
    a.pool_parents = pool_parents;
    a.factor = factor;
    a.r = r;
    a.u = u;
    a.v = v;
    a.seed = seed;
    a.seq = seq;
    a.err = w.err;
    if (insert) k_link_cut<<<blk(w.B * 32, 128), 128, 0, s>>>(a, w.B);
    else k_cut_link<<<blk(w.B * 32, 128), 128, 0, s>>>(a, w.B);
    return cudaGetLastError();
}

cudaError_t launch_scale_slots(double *w, const int64_t *slot, const double *factor, int64_t B,
                               cudaStream_t s) {
    k_scale_slots<<<blk(B, 256), 256, 0, s>>>(w, slot, factor, B);
    return cudaGetLastError();
}

cudaError_t launch_weight_rescale(double *w, const uint8_t *flag, int64_t P, double *sums,
                                  double target_flagged, double target_rest, cudaStream_t s) {
    k_weight_sums<<<1, 1024, 0, s>>>(w, flag, P, sums);
    k_weight_rescale<<<blk(P, 256), 256, 0, s>>>(w, flag, P, sums, target_flagged, target_rest);
    return cudaGetLastError();
}

cudaError_t launch_weight_sums(const double *w, const uint8_t *flag, int64_t P, double *sums,
                               cudaStream_t s) {
    k_weight_sums<<<1, 1024, 0, s>>>(w, flag, P, sums);
    return cudaGetLastError();
}

cudaError_t launch_scatter_results(const int64_t *slot, int64_t B, const int64_t *f,
                                   const int64_t *steps, const int64_t *sids, int64_t *pool_f,
                                   int64_t *pool_steps, int64_t *pool_sid, cudaStream_t s) {
    k_scatter_results<<<blk(B, 256), 256, 0, s>>>(slot, B, f, steps, sids, pool_f, pool_steps,
                                                  pool_sid);
    return cudaGetLastError();
}

}  // namespace kc
