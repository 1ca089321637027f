// Per-tree traversal passes (Algorithm 1, "vol[u] <- the volume of Sub(tau_i, u)";
// DFN of Sec. 3.2 "Implementation Details").
//
// A warp owns one tree and walks its vertices 32 at a time, so every pass costs
// one or two dependent gathers per 32 vertices instead of one per vertex.
// Dependencies inside a chunk are resolved with warp shuffles:
//   (a) bottom-up, over the parent-first order in reverse: size and volume
//       (vol = sum of degrees over the subtree).  A child inside the chunk hands
//       its total to its parent lane; a parent outside the chunk receives an
//       integer atomic add (order-independent, so results are exact).
//   (b) sibling offsets, over vertex ids ascending: among the children of one
//       parent (grouped with __match_any_sync) the offset of child c is the sum
//       of the sizes of its smaller-id siblings; a per-parent running sum
//       carries it across chunks.
//   (c) top-down, over the parent-first order: in[v] = in[p] + 1 + offset(v),
//       chains inside the chunk resolved by pointer jumping (5 rounds).
// The resulting DFN is the preorder from 0 that visits children in ascending id;
// out[v] = in[v] + size[v] - 1.  Where any valid DFN serves (f of Theorem 3
// needs only the ancestor test in[x] <= in[v] <= out[x]), (a) and (b) are
// replaced by one leaf-to-root pass of atomic reports (below).
#include <algorithm>

#include <cuda/atomic>

#include "kc_common.cuh"

namespace kc {

namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;

__device__ __forceinline__ int32_t ld_cg(const int32_t *p) { return __ldcg(p); }
__device__ __forceinline__ int64_t ld_cg(const int64_t *p) {
    return (int64_t)__ldcg((const long long *)p);
}

__global__ void __launch_bounds__(128) k_bottom_up(GraphView g, WaveView w) {
    const int lane = threadIdx.x & 31;
    const int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (t >= w.B) return;
    const int64_t n = g.n;
    const int32_t *__restrict__ ord = w.ord + wave_tree(w, t) * n;
    const uint64_t *__restrict__ word = w.word + wave_tree(w, t) * n;
    int32_t *size = w.size + t * n;
    int64_t *vol = w.vol + t * n;
    for (int64_t base = n - 1; base >= 0; base -= 32) {
        const int64_t p = base - lane;
        const bool act = p >= 0;
        int32_t v = -1, par = -2, s_own = 0;
        int64_t v_own = 0;
        if (act) {
            v = ord[p];
            par = w_next(word[v]);
            s_own = 1 + ld_cg(size + v);
            v_own = (int64_t)g.deg[v] + ld_cg(vol + v);
        }
        // lane 0 holds the latest vertex in the order; a parent always sits at a
        // higher lane than its children in the same chunk.
        bool parent_here = false;
#pragma unroll 4
        for (int j = 0; j < 32; ++j) {
            const int32_t vj = __shfl_sync(kFull, v, j);
            const int32_t pj = __shfl_sync(kFull, par, j);
            const int32_t sj = __shfl_sync(kFull, s_own, j);
            const int64_t volj = __shfl_sync(kFull, v_own, j);
            if (act && j < lane && pj == v) { s_own += sj; v_own += volj; }
            if (act && j > lane && vj == par) parent_here = true;
        }
        if (act) {
            __stcg(size + v, s_own);
            __stcg((long long *)(vol + v), (long long)v_own);
            if (par >= 0 && !parent_here) {
                atomicAdd(size + par, s_own);
                atomicAdd((unsigned long long *)(vol + par), (unsigned long long)v_own);
            }
        }
        __threadfence_block();
        __syncwarp();
    }
}

// Where any valid DFN will do, subtree sizes, volumes and sibling offsets come
// from one fully parallel pass instead of the chunked (a) + (b): every leaf
// starts a thread that reports its totals to its parent, and the thread that
// reports last continues with the parent's totals.  During the pass the walker
// word of a vertex is its report accumulator -- count of unreported children in
// the high half, sum of the reported children's sizes in the low half -- so one
// 64-bit atomic add (size in, one child out) tells a child both its offset
// among its siblings (the old size sum) and whether it reported last, and the
// last child has the parent's size without another read.  Volumes go to the
// parent with a relaxed add before that release add; the last child reads the
// parent's volume after an acquire fence.  Siblings are ordered as they
// report (the order may differ between runs; the DFN stays valid and f, sizes
// and volumes do not change).  The parent moves to din for the pass; a vertex
// writes its parent back into its word (as an in-tree word) when it reports,
// then its offset into din.  A vertex with children never has a zero word, so
// only leaves start threads.
__device__ __forceinline__ int32_t parent_of(const uint64_t *word, int64_t v) {
    return *reinterpret_cast<const int32_t *>(word + v);  // low half only
}

__global__ void k_tree_prep(GraphView g, WaveView w) {
    const int64_t n = g.n;
    const int64_t t = blockIdx.y;
    uint64_t *word = w.word + wave_tree(w, t) * n;
    int64_t *vol = w.vol + t * n;
    int32_t *din = w.din + t * n;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        din[v] = parent_of(word, v);
        word[v] = 0ull;
        vol[v] = 0;
    }
}

__global__ void k_child_count(GraphView g, WaveView w) {
    const int64_t n = g.n;
    const int64_t t = blockIdx.y;
    uint64_t *word = w.word + wave_tree(w, t) * n;
    const int32_t *din = w.din + t * n;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        const int32_t par = din[v];
        if (par >= 0 && par < n) atomicAdd((unsigned long long *)(word + par), 1ull << 32);
    }
}

__global__ void k_leaf_up(GraphView g, WaveView w) {
    const int64_t n = g.n;
    const int64_t t = blockIdx.y;
    uint64_t *word = w.word + wave_tree(w, t) * n;
    int32_t *size = w.size + t * n;
    int64_t *vol = w.vol + t * n;
    int32_t *din = w.din + t * n;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        if (*(volatile unsigned long long *)(word + v) != 0ull) continue;  // has children
        int32_t x = (int32_t)v;
        int32_t sx = 1;
        int64_t vx = (int64_t)g.deg[v];
        for (int64_t hop = 0;; ++hop) {
            if (hop > n) {  // longer than any root path: corrupt parent array
                atomicOr(w.err, kErrBadTree);
                break;
            }
            const int32_t p = din[x];
            size[x] = sx;
            vol[x] = vx;
            if (p < 0 || p >= n) {
                word[x] = w_make(-1, 0, true);
                din[x] = 0;
                if (p >= n) atomicOr(w.err, kErrBadTree);
                break;
            }
            atomicAdd((unsigned long long *)(vol + p), (unsigned long long)vx);
            cuda::atomic_ref<unsigned long long, cuda::thread_scope_device> acc(
                *reinterpret_cast<unsigned long long *>(word + p));
            const unsigned long long old =
                acc.fetch_add((unsigned long long)(uint32_t)sx - (1ull << 32),
                              cuda::memory_order_release);
            word[x] = w_make(p, 0, true);
            din[x] = (int32_t)(uint32_t)old;
            if ((old >> 32) != 1ull) break;  // siblings still to report
            cuda::atomic_thread_fence(cuda::memory_order_acquire, cuda::thread_scope_device);
            sx = 1 + (int32_t)(uint32_t)old + sx;
            vx = (int64_t)g.deg[p] + *(volatile long long *)(vol + p);
            x = p;
        }
    }
}

// Chunked alternative to the leaf-to-root pass (better for deep trees and small
// graphs): bottom-up over the parent-first order in reverse as in (a), with
// children numbered as they report to their parent -- reverse order, then lane
// order inside a chunk.  A child's offset is what an atomic add of its
// group's sizes to the parent's size returns (parent in a later chunk), or the
// parent's size at the chunk start plus the in-chunk siblings at lower lanes.
template <bool kMulti>
__global__ void __launch_bounds__(128) k_bottom_up_offsets(GraphView g_in, WaveView w_in,
                                                           MultiSub ms) {
    const int lane = threadIdx.x & 31;
    GraphView g;
    WaveView w;
    int64_t t;
    if (!pick_tree<kMulti>(ms, g_in, w_in, ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5,
                           g, w, t))
        return;
    const int64_t n = g.n;
    const int32_t *__restrict__ ord = w.ord + wave_tree(w, t) * n;
    const uint64_t *__restrict__ word = w.word + wave_tree(w, t) * n;
    int32_t *size = w.size + t * n;
    int64_t *vol = w.vol + t * n;
    int32_t *din = w.din + t * n;
    for (int64_t base = n - 1; base >= 0; base -= 32) {
        const int64_t p = base - lane;
        const bool act = p >= 0;
        int32_t v = -1, par = -2, s0 = 0, s_own = 0;
        int64_t v_own = 0;
        if (act) {
            v = ord[p];
            par = w_next(word[v]);
            s0 = ld_cg(size + v);
            s_own = 1 + s0;
            v_own = (int64_t)g.deg[v] + ld_cg(vol + v);
        }
        int plane = -1;
#pragma unroll 4
        for (int j = 0; j < 32; ++j) {
            const int32_t vj = __shfl_sync(kFull, v, j);
            const int32_t pj = __shfl_sync(kFull, par, j);
            const int32_t sj = __shfl_sync(kFull, s_own, j);
            const int64_t volj = __shfl_sync(kFull, v_own, j);
            if (act && j < lane && pj == v) { s_own += sj; v_own += volj; }
            if (act && j > lane && vj == par) plane = j;
        }
        const unsigned grp = __match_any_sync(kFull, act ? par : -3 - lane);
        int32_t excl = 0, tot = 0;
#pragma unroll 8
        for (int j = 0; j < 32; ++j) {
            const int32_t sj = __shfl_sync(kFull, s_own, j);
            if ((grp >> j) & 1u) {
                tot += sj;
                if (j < lane) excl += sj;
            }
        }
        const int leader = __ffs(grp) - 1;
        const bool out_parent = act && par >= 0 && plane < 0;
        int32_t b = 0;
        if (out_parent && lane == leader) b = atomicAdd(size + par, tot);
        b = __shfl_sync(kFull, b, leader);
        const int32_t ps0 = __shfl_sync(kFull, s0, plane >= 0 ? plane : lane);
        if (act) {
            __stcg(size + v, s_own);
            __stcg((long long *)(vol + v), (long long)v_own);
            if (out_parent)
                atomicAdd((unsigned long long *)(vol + par), (unsigned long long)v_own);
            din[v] = par < 0 ? 0 : (plane >= 0 ? ps0 : b) + excl;
        }
        __threadfence_block();
        __syncwarp();
    }
}

__global__ void __launch_bounds__(128) k_sibling_offsets(GraphView g, WaveView w) {
    const int lane = threadIdx.x & 31;
    const int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (t >= w.B) return;
    const int64_t n = g.n;
    const uint64_t *__restrict__ word = w.word + wave_tree(w, t) * n;
    const int32_t *__restrict__ size = w.size + t * n;
    int32_t *din = w.din + t * n;
    int32_t *run = w.aux + t * n;  // per-parent running sum of sizes, zeroed
    for (int64_t base = 0; base < n; base += 32) {
        const int64_t v = base + lane;
        const bool act = v < n;
        const int32_t par = act ? w_next(word[v]) : -2;
        const int32_t sz = act ? size[v] : 0;
        const unsigned grp = __match_any_sync(kFull, par);
        int32_t excl = 0, tot = 0;
#pragma unroll 8
        for (int j = 0; j < 32; ++j) {
            const int32_t sj = __shfl_sync(kFull, sz, j);
            const bool same = (grp >> j) & 1u;
            if (same) {
                tot += sj;
                if (j < lane) excl += sj;
            }
        }
        const int leader = __ffs(grp) - 1;
        int32_t basev = 0;
        if (lane == leader && par >= 0) basev = atomicAdd(run + par, tot);
        basev = __shfl_sync(kFull, basev, leader);
        if (act) din[v] = par >= 0 ? basev + excl : 0;
        __syncwarp();
    }
}

template <bool kMulti>
__global__ void __launch_bounds__(128) k_top_down(GraphView g_in, WaveView w_in, int want_pre_in,
                                                  MultiSub ms) {
    const int lane = threadIdx.x & 31;
    GraphView g;
    WaveView w;
    int64_t t;
    if (!pick_tree<kMulti>(ms, g_in, w_in, ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5,
                           g, w, t))
        return;
    const int want_pre = kMulti ? (w.bit != nullptr) : want_pre_in;
    const int64_t n = g.n;
    const int32_t *__restrict__ ord = w.ord + wave_tree(w, t) * n;
    const uint64_t *__restrict__ word = w.word + wave_tree(w, t) * n;
    int32_t *din = w.din + t * n;
    int32_t *pre = w.aux + t * n;
    // software pipeline: the order two chunks ahead and the parent and offset
    // one chunk ahead are read-only here (offsets of later chunks are not
    // overwritten before their chunk), so only in[parent] waits on the chunk
    int32_t v = -1, par = -1, off = 0;
    if (lane < n) {
        v = ord[lane];
        par = w_next(word[v]);
        off = ld_cg(din + v);
    }
    int32_t v2 = (32 + lane < n) ? ord[32 + lane] : -1;
    for (int64_t base = 0; base < n; base += 32) {
        const bool act = base + lane < n;
        // issue the next chunk's loads
        int32_t vn = v2, parn = -1, offn = 0;
        if (vn >= 0) {
            parn = w_next(word[vn]);
            offn = ld_cg(din + vn);
        }
        v2 = (base + 64 + lane < n) ? ord[base + 64 + lane] : -1;
        int ptr = -1;
#pragma unroll 8
        for (int j = 0; j < 32; ++j) {
            const int32_t vj = __shfl_sync(kFull, v, j);
            if (act && j < lane && vj == par) ptr = j;
        }
        int32_t val = 0;
        if (act && par >= 0) {
            val = 1 + off;
            if (ptr < 0) val += ld_cg(din + par);
        }
#pragma unroll
        for (int it = 0; it < 5; ++it) {
            const int src = ptr < 0 ? lane : ptr;
            const int32_t pv = __shfl_sync(kFull, val, src);
            const int pp = __shfl_sync(kFull, ptr, src);
            if (ptr >= 0) {
                val += pv;
                ptr = pp;
            }
        }
        if (act) {
            __stcg(din + v, val);
            if (want_pre && val >= 0 && val < n) pre[val] = v;
        }
        __threadfence_block();
        __syncwarp();
        v = vn;
        par = parn;
        off = offn;
    }
}

}  // namespace

cudaError_t launch_traverse(const GraphView &g, WaveView w, bool want_preorder, cudaStream_t s,
                            int *launches, int mode) {
    const size_t per = (size_t)(w.B * g.n);
    cudaError_t e;
    const unsigned blocks = (unsigned)((w.B * 32 + 127) / 128);
    const bool canonical = mode == kTravCanonical;
    if (mode == kTravChunked) {
        if ((e = cudaMemsetAsync(w.size, 0, sizeof(int32_t) * per, s)) != cudaSuccess) return e;
        if ((e = cudaMemsetAsync(w.vol, 0, sizeof(int64_t) * per, s)) != cudaSuccess) return e;
        k_bottom_up_offsets<false><<<blocks, 128, 0, s>>>(g, w, MultiSub{});
    } else if (canonical) {
        if ((e = cudaMemsetAsync(w.size, 0, sizeof(int32_t) * per, s)) != cudaSuccess) return e;
        if ((e = cudaMemsetAsync(w.vol, 0, sizeof(int64_t) * per, s)) != cudaSuccess) return e;
        // children in ascending id (the DFN the oracle and the update kernels use)
        if ((e = cudaMemsetAsync(w.aux, 0, sizeof(int32_t) * per, s)) != cudaSuccess) return e;
        k_bottom_up<<<blocks, 128, 0, s>>>(g, w);
        k_sibling_offsets<<<blocks, 128, 0, s>>>(g, w);
    } else {
        const dim3 grid((unsigned)std::min<int64_t>((g.n + 255) / 256, 1024), (unsigned)w.B);
        k_tree_prep<<<grid, 256, 0, s>>>(g, w);
        k_child_count<<<grid, 256, 0, s>>>(g, w);
        k_leaf_up<<<grid, 256, 0, s>>>(g, w);
    }
    k_top_down<false><<<blocks, 128, 0, s>>>(g, w, want_preorder ? 1 : 0, MultiSub{});
    if (launches) *launches += canonical ? 3 : (mode == kTravChunked ? 2 : 4);
    return cudaGetLastError();
}

cudaError_t launch_traverse_multi(const MultiSub &ms, cudaStream_t s) {
    if (ms.count <= 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((ms.count * 32 + 127) / 128);
    k_bottom_up_offsets<true><<<blocks, 128, 0, s>>>(GraphView{}, WaveView{}, ms);
    k_top_down<true><<<blocks, 128, 0, s>>>(GraphView{}, WaveView{}, 0, ms);
    return cudaGetLastError();
}

}  // namespace kc
