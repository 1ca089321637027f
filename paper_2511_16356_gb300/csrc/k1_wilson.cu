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
    int32_t pos = 1;       // ord[0] = root
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
            const VRec rv = rec[v];
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

}  // namespace

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
