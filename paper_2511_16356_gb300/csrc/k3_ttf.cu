// f(tau) of Theorem 3 for every tree of a wave (Sec. 3.2).
//
// With p(x) the tau parent, p0(x) the tau0 parent and vol(x) = vol(Sub(tau, x)),
//   f(tau) = sum_{v != r} d(v) Q(v),
//   Q(v)   = sum over tau-ancestors x of v (x != r, x included when x = v) of
//              [p(x) = p0(x)]  [v in Sub(tau0, x)]    (2m - vol(x))      (forward)
//            - [p0(p(x)) = x]  [v in Sub(tau0, p(x))] (2m - vol(x))      (reverse)
// (Theorem 4 with the d(u) weight of Algorithm 1 and the reverse undo written as
// the negation of its add).  Two kernels evaluate it:
//
//  SCAN: for each v, walk up tau0 (at most its depth: ecc(r) for the BFS tree)
//        and test tau-ancestry with the DFN intervals of tau: O(n ecc) work, all
//        vertices of all trees in parallel.  Used when the depth is small (the
//        O(n Delta) bound of Thm 8).
//  BIT:  Algorithm 1: a DFS over tau in preorder keeps, for the tau-ancestors of
//        the current vertex, range adds over tau0-DFN intervals in a Fenwick
//        array and queries the point in0(v).  O(n log n) per tree.  A warp owns a
//        tree and handles 32 preorder positions per round: all 32 point queries
//        are loaded first, then the 32 visits are replayed in lane order with the
//        stack held in registers, each range add both issued to the Fenwick array
//        (integer atomics) and folded into the pending queries of later lanes.
// Both are templates: the batched instances take (graph, tree) entries and
// per-graph tables, so trees of many graphs share one launch.
#include <algorithm>

#include "kc_common.cuh"

namespace kc {

namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;

template <bool kMulti>
__global__ void __launch_bounds__(256) k_ttf_scan(GraphView g_in, WaveView w_in, MultiSub ms) {
    GraphView g;
    WaveView w;
    int64_t t;
    if (!pick_tree<kMulti>(ms, g_in, w_in, blockIdx.y, g, w, t)) return;  // whole block
    const int64_t n = g.n;
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t *__restrict__ word = w.word + wave_tree(w, t) * n;
    const int32_t *__restrict__ din = w.din + t * n;
    const int32_t *__restrict__ size = w.size + t * n;
    const int64_t *__restrict__ vol = w.vol + t * n;
    const int32_t r = g.root;
    const int64_t twom = g.twom;
    long long contrib = 0;
    if (v < n && v != r) {
        const int32_t inv = din[v];
        long long q = 0;
        int32_t x = (int32_t)v;
        for (int it = 0; x != r && it <= g.ecc; ++it) {
            const int32_t p0x = g.p0[x];
            const int32_t px = w_next(word[x]);
            if (px == p0x) {
                const int32_t inx = din[x];
                if (inx <= inv && inv <= inx + size[x] - 1) q += twom - vol[x];
            } else if (p0x != r && w_next(word[p0x]) == x) {
                const int32_t inw = din[p0x];
                if (inw <= inv && inv <= inw + size[p0x] - 1) q -= twom - vol[p0x];
            }
            x = p0x;
        }
        contrib = (long long)g.deg[v] * q;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) contrib += __shfl_down_sync(kFull, contrib, o);
    __shared__ long long part[8];
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = contrib;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long s = 0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += part[k];
        if (s != 0) atomicAdd((unsigned long long *)(w.f + wave_tree(w, t)), (unsigned long long)s);
    }
}

// Fenwick point update at 1-based index i, the warp's lanes sharing the chain.
// With j = i - 1 the chain is j, j | (j + 1), ...: its k-th node sets the k
// lowest zero bits of j, i.e. equals j | (2^(b+1) - 1) where b is the k-th
// zero bit.  So lane b (b < 31) owns the node of zero bit b of j and lane 31
// owns node 0 (j itself); every node is visited exactly once.
__device__ __forceinline__ void bit_point_add(int64_t *bit, int64_t n, int lane, int64_t i,
                                              long long val) {
    const uint32_t j = (uint32_t)(i - 1);  // host guarantees n < 2^31
    int64_t node;
    if (lane == 31) node = (int64_t)j + 1;
    else if ((j >> lane) & 1u) node = -1;
    else node = (int64_t)(j | ((2u << lane) - 1u)) + 1;
    if (node >= 1 && node <= n) atomicAdd((unsigned long long *)(bit + node), (unsigned long long)val);
}

// range add [l, r] (0-based positions) += val, as two point updates
__device__ __forceinline__ void bit_range_add(int64_t *bit, int64_t n, int lane, int32_t l,
                                              int32_t r, long long val) {
    bit_point_add(bit, n, lane, (int64_t)l + 1, val);
    if ((int64_t)r + 2 <= n) bit_point_add(bit, n, lane, (int64_t)r + 2, -val);
}

// Range add of tau-ancestor x (x != r, tau parent par) in Algorithm 1: kind 1
// when p(x) = p0(x) (tau0-subtree of x, value 2m - vol(x)), kind 2 when
// p0(p(x)) = x (tau0-subtree of p(x), value vol(x) - 2m), 0 otherwise.
__device__ __forceinline__ int ttf_entry(const GraphView &g, int32_t x, int32_t par, int32_t r,
                                         int32_t twom, int64_t volx, int32_t &el, int32_t &er,
                                         int32_t &eval) {
    const int32_t vv = (int32_t)volx;
    if (g.p0[x] == par) {
        el = g.in0[x]; er = g.out0[x]; eval = twom - vv;
        return 1;
    }
    if (par != r && g.p0[par] == x) {
        el = g.in0[par]; er = g.out0[par]; eval = vv - twom;
        return 2;
    }
    return 0;
}

// One warp replays the preorder positions [lo, hi) of sub-wave tree t
// (Algorithm 1) on the Fenwick array `bit` (1-based) and the memory stack `stk`
// (sp entries on entry, the deepest on top); returns this lane's share of the
// sum of d(v) Q(v) over those positions.  ok = false on a stack overflow (the
// error bit is set).
__device__ __forceinline__ long long ttf_bit_sweep(const GraphView &g, const WaveView &w,
                                                   int64_t t, int64_t *bit, int4 *stk,
                                                   int64_t lo, int64_t hi, int64_t sp,
                                                   bool &ok) {
    const int lane = threadIdx.x & 31;
    const int64_t n = g.n;
    const int32_t r = g.root;
    const int32_t twom = (int32_t)g.twom;  // host guarantees 2m < 2^31 for this kernel
    const uint64_t *__restrict__ word = w.word + wave_tree(w, t) * n;
    const int32_t *__restrict__ size = w.size + t * n;
    const int64_t *__restrict__ vol = w.vol + t * n;
    const int32_t *__restrict__ pre = w.aux + t * n;
    const unsigned lt_mask = (1u << lane) - 1u;
    ok = true;

    long long facc = 0;     // this lane's share of f
    for (int64_t base = lo; base < hi; base += 32) {
        const int64_t i = base + lane;
        const bool act = i < hi;
        // ---- per-vertex data for preorder position i
        int32_t v = -1, kind = 0, el = 0, er = 0, eval = 0, eout = 0, qpos = 0, dv = 0;
        if (act) {
            v = pre[i];
            if (v < 0 || v >= n) {  // preorder is a permutation; anything else is corrupt
                atomicOr(w.err, kErrBadTree);
                v = r;
            }
            const int32_t par = w_next(word[v]);
            qpos = g.in0[v];
            dv = g.deg[v];
            eout = (int32_t)i + size[v] - 1;
            if (v != r) kind = ttf_entry(g, v, par, r, twom, vol[v], el, er, eval);
        }
        // ---- prefix sums at the start of the chunk
        long long pf = 0;
        if (act) {
            for (int64_t k = (int64_t)qpos + 1; k > 0; k &= k - 1)
                pf += __ldcg((const long long *)(bit + k));
        }
        // every query load must have returned before this chunk issues its own
        // atomics: reading pf in a shuffle makes the warp wait for them
        pf = __shfl_sync(kFull, pf, lane);
        long long corr = 0;
        // ---- top of the memory stack, one entry per lane (lane k: entry sp-1-k)
        int64_t mbase = sp;   // window covers entries [mbase - 32, mbase)
        int4 win = make_int4(0, 0, 0, 0);
        if (mbase - 1 - lane >= 0) win = stk[mbase - 1 - lane];
        int mtop = 0;         // entries of the window already popped
        int64_t mpopped = 0;  // memory entries popped in this chunk
        unsigned cmask = 0;   // chunk entries alive on the stack (push order = lane order)
        __syncwarp();
        for (int j = 0; j < 32; ++j) {
            const int64_t ij = base + j;
            if (ij >= hi) break;
            // pop every stacked ancestor whose subtree ended before position ij
            while (true) {
                int32_t pl, pr, pv;
                if (cmask) {
                    const int h = 31 - __clz(cmask);
                    const int32_t o = __shfl_sync(kFull, eout, h);
                    if (o >= ij) break;
                    pl = __shfl_sync(kFull, el, h);
                    pr = __shfl_sync(kFull, er, h);
                    pv = __shfl_sync(kFull, eval, h);
                    cmask &= ~(1u << h);
                } else {
                    if (sp - mpopped <= 0) break;
                    if (mtop == 32) {  // reload the window below what was consumed
                        mbase = sp - mpopped;
                        win = make_int4(0, 0, 0, 0);
                        if (mbase - 1 - lane >= 0) win = stk[mbase - 1 - lane];
                        mtop = 0;
                    }
                    const int32_t o = __shfl_sync(kFull, win.x, mtop);
                    if (o >= ij) break;
                    pl = __shfl_sync(kFull, win.y, mtop);
                    pr = __shfl_sync(kFull, win.z, mtop);
                    pv = __shfl_sync(kFull, win.w, mtop);
                    ++mtop;
                    ++mpopped;
                }
                // undo: add the negation
                bit_range_add(bit, n, lane, pl, pr, -(long long)pv);
                if (lane >= j && pl <= qpos && qpos <= pr) corr -= pv;
            }
            const int kj = __shfl_sync(kFull, kind, j);
            if (kj) {
                const int32_t l = __shfl_sync(kFull, el, j);
                const int32_t rr = __shfl_sync(kFull, er, j);
                const int32_t val = __shfl_sync(kFull, eval, j);
                bit_range_add(bit, n, lane, l, rr, (long long)val);
                if (lane >= j && l <= qpos && qpos <= rr) corr += val;
                cmask |= 1u << j;
            }
        }
        if (act) facc += (long long)dv * (pf + corr);
        // ---- spill the surviving chunk entries on top of the memory stack
        const int64_t nsp = sp - mpopped;
        if ((cmask >> lane) & 1u) {
            const int64_t slot = nsp + __popc(cmask & lt_mask);
            if (slot < w.stack_cap) stk[slot] = make_int4(eout, el, er, eval);
        }
        sp = nsp + __popc(cmask);
        if (sp > w.stack_cap) {
            if (lane == 0) atomicOr(w.err, kErrBadTree);
            ok = false;
            return 0;
        }
        __threadfence_block();
        __syncwarp();
    }
    return facc;
}

template <bool kMulti>
__global__ void __launch_bounds__(128) k_ttf_bit(GraphView g_in, WaveView w_in, MultiSub ms) {
    const int lane = threadIdx.x & 31;
    GraphView g;
    WaveView w;
    int64_t t;
    if (!pick_tree<kMulti>(ms, g_in, w_in, ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5,
                           g, w, t))
        return;
    const int64_t n = g.n;
    int64_t *bit = w.bit + t * (n + 1);  // zeroed, 1-based
    int4 *stk = reinterpret_cast<int4 *>(w.stack) + t * w.stack_cap;
    bool ok;
    long long facc = ttf_bit_sweep(g, w, t, bit, stk, 0, n, 0, ok);
    if (!ok) return;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) facc += __shfl_down_sync(kFull, facc, o);
    if (lane == 0) w.f[wave_tree(w, t)] = facc;
}

// Algorithm 1 over one preorder segment [lo, hi) of a tree per warp.  At
// position lo the DFS stack holds the strict tau-ancestors of u = pre[lo] that
// add a range, and the Fenwick array holds the sum of their range adds (every
// ancestor of a later position that precedes lo is an ancestor of u; entries
// pushed and popped before lo cancel).  Lane 0 collects them walking up the
// tau parents (deepest first), the warp reverses them into stack order (root
// side at the bottom) and replays their range adds, then sweeps the segment;
// its share of f is added to the tree's f, which the caller zeroed.
__global__ void __launch_bounds__(128) k_ttf_bit_seg(GraphView g, WaveView w,
                                                     const TtfSeg *__restrict__ segs,
                                                     int64_t nseg) {
    const int lane = threadIdx.x & 31;
    const int64_t si = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (si >= nseg) return;
    const TtfSeg sg = segs[si];
    const int64_t n = g.n;
    const int32_t r = g.root;
    const int32_t twom = (int32_t)g.twom;
    const int64_t t = sg.t;
    const uint64_t *__restrict__ word = w.word + wave_tree(w, t) * n;
    const int32_t *__restrict__ size = w.size + t * n;
    const int64_t *__restrict__ vol = w.vol + t * n;
    const int32_t *__restrict__ din = w.din + t * n;
    const int32_t *__restrict__ pre = w.aux + t * n;
    int4 *stk = sg.stk;
    int64_t sp = 0;
    if (sg.lo > 0) {
        long long cnt = 0;
        if (lane == 0) {
            const int32_t u = pre[sg.lo];
            int32_t x = (u >= 0 && u < n) ? w_next(word[u]) : -1;
            if (u < 0 || u >= n) cnt = -1;
            int64_t hops = 0;
            while (cnt >= 0 && x != r) {
                if (x < 0 || x >= n || ++hops > n) {
                    cnt = -1;
                    break;
                }
                const int32_t par = w_next(word[x]);
                if (par < 0 || par >= n) {  // only the root has no parent
                    cnt = -1;
                    break;
                }
                int32_t el = 0, er = 0, eval = 0;
                if (ttf_entry(g, x, par, r, twom, vol[x], el, er, eval)) {
                    if (cnt >= w.stack_cap) {
                        cnt = -1;
                        break;
                    }
                    stk[cnt++] = make_int4(din[x] + size[x] - 1, el, er, eval);
                }
                x = par;
            }
            if (cnt < 0) atomicOr(w.err, kErrBadTree);
        }
        cnt = __shfl_sync(kFull, cnt, 0);
        if (cnt < 0) return;
        __syncwarp();
        for (long long e = lane; e < cnt / 2; e += 32) {
            const int4 a = stk[e], b = stk[cnt - 1 - e];
            stk[e] = b;
            stk[cnt - 1 - e] = a;
        }
        __syncwarp();
        for (long long e = 0; e < cnt; ++e) {
            const int4 en = stk[e];
            bit_range_add(sg.bit, n, lane, en.y, en.z, (long long)en.w);
        }
        __threadfence_block();
        __syncwarp();
        sp = cnt;
    }
    bool ok;
    long long facc = ttf_bit_sweep(g, w, t, sg.bit, stk, sg.lo, sg.hi, sp, ok);
    if (!ok) return;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) facc += __shfl_down_sync(kFull, facc, o);
    if (lane == 0 && facc != 0)
        atomicAdd((unsigned long long *)(w.f + wave_tree(w, t)), (unsigned long long)facc);
}

// zero entries 1 .. n of every segment's Fenwick array
__global__ void k_zero_seg_bits(const TtfSeg *__restrict__ segs, int64_t nseg, int64_t n) {
    for (int64_t s = blockIdx.y; s < nseg; s += gridDim.y) {
        int64_t *b = segs[s].bit;
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
             i += (int64_t)gridDim.x * blockDim.x)
            b[i + 1] = 0;
    }
}

}  // namespace

cudaError_t launch_ttf_scan(const GraphView &g, WaveView w, cudaStream_t s) {
    if (!w.tmap) {  // with a tree map the caller has zeroed f for the whole wave
        cudaError_t e = cudaMemsetAsync(w.f, 0, sizeof(int64_t) * (size_t)w.B, s);
        if (e != cudaSuccess) return e;
    }
    dim3 grid((unsigned)((g.n + 255) / 256), (unsigned)w.B);
    k_ttf_scan<false><<<grid, 256, 0, s>>>(g, w, MultiSub{});
    return cudaGetLastError();
}

cudaError_t launch_ttf_bit_seg(const GraphView &g, WaveView w, const TtfSeg *segs, int64_t nseg,
                              cudaStream_t s) {
    if (nseg <= 0) return cudaSuccess;
    const dim3 zgrid((unsigned)std::min<int64_t>((g.n + 255) / 256, 64),
                     (unsigned)std::min<int64_t>(nseg, 65535));
    k_zero_seg_bits<<<zgrid, 256, 0, s>>>(segs, nseg, g.n);
    k_ttf_bit_seg<<<(unsigned)((nseg * 32 + 127) / 128), 128, 0, s>>>(g, w, segs, nseg);
    return cudaGetLastError();
}

cudaError_t launch_ttf_bit(const GraphView &g, WaveView w, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(w.bit, 0, sizeof(int64_t) * (size_t)(w.B * (g.n + 1)), s);
    if (e != cudaSuccess) return e;
    k_ttf_bit<false><<<(unsigned)((w.B * 32 + 127) / 128), 128, 0, s>>>(g, w, MultiSub{});
    return cudaGetLastError();
}

cudaError_t launch_ttf_scan_multi(const MultiSub &ms, int64_t max_n, cudaStream_t s) {
    for (int64_t r0 = 0; r0 < ms.count; r0 += 65535) {  // grid rows: at most 65535
        MultiSub part = ms;
        part.entry = ms.entry + r0;
        part.count = std::min<int64_t>(65535, ms.count - r0);
        dim3 grid((unsigned)((max_n + 255) / 256), (unsigned)part.count);
        k_ttf_scan<true><<<grid, 256, 0, s>>>(GraphView{}, WaveView{}, part);
    }
    return cudaGetLastError();
}

cudaError_t launch_ttf_bit_multi(const MultiSub &ms, cudaStream_t s) {
    if (ms.count <= 0) return cudaSuccess;
    k_ttf_bit<true><<<(unsigned)((ms.count * 32 + 127) / 128), 128, 0, s>>>(GraphView{},
                                                                           WaveView{}, ms);
    return cudaGetLastError();
}

}  // namespace kc
