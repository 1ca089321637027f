// Sample pool maintenance and the cross-tree reduction of Algorithm 1's last
// line (K_hat = sum f / (2m omega)) and of Algorithm 3's weighted sum.
//
// The pool holds, per tree: f (int64, exact), weight w (FP64; 1 for freshly
// sampled trees), Wilson step count, sample id and, when trees are retained,
// the parent array.  The reduction runs in one block with a fixed partition
// and a fixed combining tree, so its result is bit-reproducible; the sum of f
// is exact (128-bit integer in two 64-bit limbs).
#include "kc_common.cuh"

namespace kc {

namespace {

__global__ void k_pool_append(WaveView w, int64_t first, int64_t *pool_f, double *pool_w,
                              int64_t *pool_steps, int64_t *pool_sid, const int64_t *sids) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= w.B) return;
    pool_f[first + t] = w.f[t];
    pool_w[first + t] = 1.0;
    pool_steps[first + t] = w.steps[t];
    pool_sid[first + t] = sids[t];
}

__global__ void k_pool_parents(const uint64_t *word, int64_t B, int64_t n, int32_t *dst) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < B * n) dst[k] = w_next(word[k]);
}

__global__ void k_words_from_parents(int64_t n, int64_t B, const int32_t *parents,
                                     uint64_t *word) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < B * n) word[k] = w_make(parents[k], 0, false);
}

struct I128 {
    long long hi;
    unsigned long long lo;
};
__device__ __forceinline__ void add_i64(I128 &a, long long x) {
    const unsigned long long old = a.lo;
    a.lo += (unsigned long long)x;
    a.hi += (x < 0 ? -1LL : 0LL) + (a.lo < old ? 1LL : 0LL);
}
__device__ __forceinline__ void add_i128(I128 &a, const I128 &b) {
    const unsigned long long old = a.lo;
    a.lo += b.lo;
    a.hi += b.hi + (a.lo < old ? 1LL : 0LL);
}

__global__ void __launch_bounds__(1024) k_pool_reduce(const int64_t *f, const double *w,
                                                      int64_t count, double inv_twom,
                                                      PoolSums *out) {
    __shared__ I128 s_i[1024];
    __shared__ double s_wf[1024], s_w[1024], s_x2[1024];
    const int tid = threadIdx.x;
    I128 acc{0, 0};
    double wf = 0.0, ws = 0.0, x2 = 0.0;
    for (int64_t k = tid; k < count; k += blockDim.x) {
        const long long fk = (long long)f[k];
        const double wk = w[k];
        add_i64(acc, fk);
        const double x = (double)fk * inv_twom;
        wf += wk * x;
        ws += wk;
        x2 += x * x;
    }
    s_i[tid] = acc;
    s_wf[tid] = wf;
    s_w[tid] = ws;
    s_x2[tid] = x2;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if (tid < h) {
            add_i128(s_i[tid], s_i[tid + h]);
            s_wf[tid] += s_wf[tid + h];
            s_w[tid] += s_w[tid + h];
            s_x2[tid] += s_x2[tid + h];
        }
        __syncthreads();
    }
    if (tid == 0) {
        out->f_hi = s_i[0].hi;
        out->f_lo = s_i[0].lo;
        out->wf = s_wf[0];
        out->w = s_w[0];
        out->x2 = s_x2[0];
        out->count = count;
    }
}

__global__ void k_out_from_size(int64_t n, const int32_t *din, const int32_t *size,
                                int32_t *dout) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n) dout[v] = din[v] + size[v] - 1;
}

__global__ void k_iota(int64_t *dst, int64_t start, int64_t count) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < count) dst[k] = start + k;
}

}  // namespace

cudaError_t launch_iota(int64_t *dst, int64_t start, int64_t count, cudaStream_t s) {
    k_iota<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(dst, start, count);
    return cudaGetLastError();
}

cudaError_t launch_pool_append(WaveView w, int64_t first, int64_t *pool_f, double *pool_w,
                               int64_t *pool_steps, int64_t *pool_sid, const int64_t *sids,
                               int32_t *pool_parents, int64_t n, cudaStream_t s) {
    k_pool_append<<<(unsigned)((w.B + 255) / 256), 256, 0, s>>>(w, first, pool_f, pool_w,
                                                               pool_steps, pool_sid, sids);
    if (pool_parents) {
        const int64_t tot = w.B * n;
        k_pool_parents<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(w.word, w.B, n,
                                                                    pool_parents + first * n);
    }
    return cudaGetLastError();
}

cudaError_t launch_pool_reduce(const int64_t *f, const double *w, int64_t count, int64_t twom,
                               void *scratch, cudaStream_t s) {
    k_pool_reduce<<<1, 1024, 0, s>>>(f, w, count, 1.0 / (double)twom,
                                     reinterpret_cast<PoolSums *>(scratch));
    return cudaGetLastError();
}

cudaError_t launch_words_from_parents(int64_t n, int64_t B, const int32_t *parents,
                                      uint64_t *word, cudaStream_t s) {
    const int64_t tot = B * n;
    k_words_from_parents<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(n, B, parents, word);
    return cudaGetLastError();
}

cudaError_t launch_out_from_size(int64_t n, const int32_t *din, const int32_t *size,
                                 int32_t *dout, cudaStream_t s) {
    k_out_from_size<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, din, size, dout);
    return cudaGetLastError();
}

}  // namespace kc
