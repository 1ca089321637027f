// kc_wilson_noalloc: Wilson spanning-tree sampling that allocates nothing.
//
// Some callers cannot call cudaMalloc at the point where they need trees:
// code running inside a custom allocator or a memory-pool callback, plugins
// that are handed a fixed device budget by their host application, and
// real-time paths that must not hit the driver's allocator (its latency is
// unbounded and it may synchronise the device).  This entry point takes every
// input and output as caller-owned device memory and keeps its only working
// state -- one 8-byte walker word per vertex per tree -- in the fixed array
// below, which every GPU that loads this library holds until the process
// exits.
//
// Limits and sharing: the array holds kNoAllocWords words (64 MiB), so a call
// needs n * n_trees <= kNoAllocWords; larger requests are rejected with
// KC_ERR_SCRATCH_LIMIT.  Every call on a device reuses the same array and leaves
// the last call's contents in it; each call clears the part it uses first.
// Calls that overlap on the GPU (two streams, or two host threads) race on
// the array and produce garbage: serialise them.
#include <algorithm>
#include <mutex>

#include "kc_common.cuh"

namespace kc {
namespace {

constexpr int64_t kNoAllocWords = (int64_t)8 << 20;  // 8 Mi words = 64 MiB
constexpr int kMaxDevices = 64;

// The scratch: walker words of the trees of one call, tree-major.
static __device__ __align__(256) uint64_t g_noalloc_words[kNoAllocWords];

// Host-side device addresses of g_noalloc_words, one per device (resolved on
// the first call made with that device current).
uint64_t *g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

// One lane per tree, straight from the CSR (no walk records): the same
// arrows (vertex u leaves along neighbour bounded(seed, u, k, sample, WALK,
// deg u) on its k-th departure) and hence the same trees and step counts as
// the library's other samplers.
__global__ void __launch_bounds__(128)
k_wilson_noalloc(int64_t n, const int64_t *__restrict__ row_off, const int32_t *__restrict__ col,
                 int32_t root, uint64_t seed, int64_t first_id, int64_t n_trees,
                 uint64_t *scratch, int32_t *__restrict__ parent, int64_t *__restrict__ steps_out,
                 int64_t step_cap, uint32_t *__restrict__ status) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_trees) return;
    uint64_t *word = scratch + t * n;
    const uint32_t sample = (uint32_t)(first_id + t);
    word[root] = w_make(-1, 0, true);
    int64_t steps = 0;
    bool ok = true;
    for (int64_t s = 0; s < n && ok; ++s) {
        if (w_in_tree(word[s])) continue;
        int32_t u = (int32_t)s;
        uint64_t wu = word[u];
        while (!w_in_tree(wu)) {
            const int64_t off = row_off[u];
            const uint32_t d = (uint32_t)(row_off[u + 1] - off);
            const uint32_t k = bounded_draw(seed, (uint32_t)u, w_count(wu), sample, kTagWalk, d);
            const int32_t v = col[off + k];
            word[u] = w_make(v, w_count(wu) + 1, false);
            // the library's samplers stop at 2^25 departures of one vertex (the
            // 32-walker word packs the count in 25 bits); stopping here too keeps
            // the contract identical and the 31-bit field from wrapping
            if (++steps > step_cap || w_count(wu) + 1 >= (1u << 25)) {
                ok = false;
                break;
            }
            u = v;
            wu = word[u];
        }
        if (!ok) break;
        for (int32_t x = (int32_t)s; !w_in_tree(word[x]);) {
            const uint64_t wx = word[x];
            word[x] = w_make(w_next(wx), 0, true);
            x = w_next(wx);
        }
    }
    if (!ok) atomicOr(status, 1u);
    int32_t *par = parent + t * n;
    for (int64_t v = 0; v < n; ++v) par[v] = v == root ? -1 : w_next(word[v]);
    steps_out[t] = steps;
}

}  // namespace
}  // namespace kc

extern "C" kc_status kc_wilson_noalloc(int64_t n, const int64_t *d_row_off, const int32_t *d_col,
                                       int32_t root, uint64_t seed, int64_t first_sample_id,
                                       int64_t n_trees, int64_t step_cap, int32_t *d_parent,
                                       int64_t *d_steps, uint32_t *d_status, void *stream) {
    using namespace kc;
    // sample ids are 32-bit: first_sample_id + n_trees <= 2^32, checked without
    // forming the sum of two unchecked values
    if (n < 2 || n_trees < 0 || !d_row_off || !d_col || !d_parent || !d_steps || !d_status ||
        root < 0 || root >= n || first_sample_id < 0 || first_sample_id > ((int64_t)1 << 32) ||
        n_trees > ((int64_t)1 << 32) - first_sample_id)
        return KC_ERR_INVALID_ARG;
    if (n_trees == 0) return KC_OK;
    if (n > kNoAllocWords / n_trees) return KC_ERR_SCRATCH_LIMIT;
    // the launch check below reads the thread's last error: clear one that an
    // earlier, unrelated runtime call left pending
    (void)cudaGetLastError();
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        (void)cudaGetLastError();
        return KC_ERR_NO_DEVICE;
    }
    uint64_t *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_scratch_mu);
        if (!g_scratch_addr[dev]) {
            void *p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_words);
            if (e != cudaSuccess || !p) {
                (void)cudaGetLastError();
                return KC_ERR_CUDA;
            }
            g_scratch_addr[dev] = (uint64_t *)p;
        }
        scratch = g_scratch_addr[dev];
    }
    cudaStream_t s = (cudaStream_t)stream;
    // the words of this call's trees must start at zero (free, no departures)
    if (cudaMemsetAsync(scratch, 0, sizeof(uint64_t) * (size_t)(n * n_trees), s) != cudaSuccess ||
        cudaMemsetAsync(d_status, 0, sizeof(uint32_t), s) != cudaSuccess) {
        (void)cudaGetLastError();
        return KC_ERR_CUDA;
    }
    const int64_t cap = step_cap > 0 ? step_cap : std::max<int64_t>((int64_t)1 << 22, 1024 * n);
    k_wilson_noalloc<<<(unsigned)((n_trees + 127) / 128), 128, 0, s>>>(
        n, d_row_off, d_col, root, seed, first_sample_id, n_trees, scratch, d_parent, d_steps, cap,
        d_status);
    if (cudaGetLastError() != cudaSuccess) return KC_ERR_CUDA;
    return KC_OK;
}
