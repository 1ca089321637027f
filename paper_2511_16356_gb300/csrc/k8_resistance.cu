// Effective resistance R(u, v) = (e_u - e_v)^T L^+ (e_u - e_v) of an edge, needed
// by the insertion cases of Algorithms 2 and 3 ("Compute R(u, v) in G + (u, v)").
// The paper uses an approximate single-pair method; here it is the solution of
// L x = e_u - e_v by conjugate gradients in FP64 with the Jacobi (degree)
// preconditioner, R = x_u - x_v.  L is singular but the right-hand side is
// orthogonal to its null space, so the iteration stays consistent.  Dot
// products use a fixed two-level reduction, so R is bit-reproducible.
#include "kc_common.cuh"

namespace kc {
namespace {

constexpr int kBlocks = 304;   // 2 per SM
constexpr int kThreads = 256;

__global__ void k_lap_spmv(GraphView g, const double *p, double *out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.n) return;
    double acc = (double)g.deg[i] * p[i];
    for (int64_t e = g.row_off[i]; e < g.row_off[i + 1]; ++e) acc -= p[g.col[e]];
    out[i] = acc;
}

// partial[b] = sum over this block's grid-stride share of a_i * b_i
__global__ void __launch_bounds__(kThreads) k_dot_partial(int64_t n, const double *a,
                                                          const double *b, double *partial) {
    __shared__ double sh[kThreads];
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        acc += a[i] * b[i];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) sh[threadIdx.x] += sh[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

__global__ void k_dot_final(const double *partial, int nb, double *out) {
    __shared__ double sh[512];
    double acc = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) acc += partial[i];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) sh[threadIdx.x] += sh[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0];
}

// x += alpha p ; r -= alpha Ap ; z = r / d     (alpha = s[0] / s[1])
__global__ void k_cg_update_xr(int64_t n, const int32_t *deg, const double *sc, double *x,
                               double *r, double *z, const double *p, const double *ap) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double alpha = sc[0] / sc[1];
    x[i] += alpha * p[i];
    const double ri = r[i] - alpha * ap[i];
    r[i] = ri;
    z[i] = ri / (double)deg[i];
}

// p = z + beta p   (beta = s[2] / s[0], new rz over old rz)
__global__ void k_cg_update_p(int64_t n, const double *sc, const double *z, double *p) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    p[i] = z[i] + (sc[2] / sc[0]) * p[i];
}

__global__ void k_cg_init(int64_t n, const int32_t *deg, int32_t u, int32_t v, double *x, double *r,
                          double *z, double *p) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double b = (i == u) ? 1.0 : ((i == v) ? -1.0 : 0.0);
    x[i] = 0.0;
    r[i] = b;
    z[i] = b / (double)deg[i];
    p[i] = z[i];
}

}  // namespace

size_t cg_scratch_doubles(int64_t n) { return (size_t)(5 * n + kBlocks + 8); }

void cg_graph_release(CgGraph &c) {
    if (c.exec) cudaGraphExecDestroy(c.exec);
    if (c.capture_stream) cudaStreamDestroy(c.capture_stream);
    c = CgGraph{};
}

cudaError_t resistance_cg(const GraphView &g, int32_t u, int32_t v, double tol, int64_t max_iter,
                          double *buf, double *R_out, int64_t *iters_out, int *launches,
                          cudaStream_t s, CgGraph *cache) {
    const int64_t n = g.n;
    cudaError_t e = cudaSuccess;
    double *x = buf, *r = x + n, *z = r + n, *p = z + n, *ap = p + n, *part = ap + n,
           *sc = part + kBlocks;  // sc[0] = rz, sc[1] = pAp, sc[2] = rz_new, sc[3] = rr
    const unsigned nb = (unsigned)((n + kThreads - 1) / kThreads);
    int nl = 0;
    cudaStream_t cur = s;  // the stream the helpers below enqueue on
    auto dot = [&](const double *a, const double *b, double *out) {
        k_dot_partial<<<kBlocks, kThreads, 0, cur>>>(n, a, b, part);
        k_dot_final<<<1, 512, 0, cur>>>(part, kBlocks, out);
        nl += 2;
    };
    k_cg_init<<<nb, kThreads, 0, s>>>(n, g.deg, u, v, x, r, z, p);
    ++nl;
    dot(r, z, sc + 0);
    // one CG iteration: 9 launches and a scalar copy, all on s
    auto iteration = [&]() -> cudaError_t {
        k_lap_spmv<<<nb, kThreads, 0, cur>>>(g, p, ap);
        ++nl;
        dot(p, ap, sc + 1);
        k_cg_update_xr<<<nb, kThreads, 0, cur>>>(n, g.deg, sc, x, r, z, p, ap);
        ++nl;
        dot(r, z, sc + 2);
        dot(r, r, sc + 3);
        k_cg_update_p<<<nb, kThreads, 0, cur>>>(n, sc, z, p);
        ++nl;
        return cudaMemcpyAsync(sc + 0, sc + 2, sizeof(double), cudaMemcpyDeviceToDevice, cur);
    };
    // The residual is checked every kChunk iterations.  With a cache, the
    // chunk's launches are captured once into a CUDA graph (the vectors, the
    // CSR and n are its key) and replayed as one launch per chunk.
    constexpr int kChunk = 8;
    const void *key[5] = {g.row_off, g.col, g.deg, buf, (const void *)(intptr_t)n};
    if (cache && cache->exec) {
        bool same = true;
        for (int k = 0; k < 5; ++k) same = same && cache->key[k] == key[k];
        if (!same) {
            cudaGraphExecDestroy(cache->exec);
            cache->exec = nullptr;
        }
    }
    if (cache && !cache->exec && max_iter >= kChunk) {
        // captured on a private stream (the caller's may be the legacy default
        // stream, which cannot be captured); replayed on s
        if (!cache->capture_stream &&
            (e = cudaStreamCreateWithFlags(&cache->capture_stream, cudaStreamNonBlocking)) !=
                cudaSuccess)
            return e;
        cudaGraph_t graph = nullptr;
        cur = cache->capture_stream;
        e = cudaStreamBeginCapture(cur, cudaStreamCaptureModeThreadLocal);
        const int nl0 = nl;
        for (int k = 0; k < kChunk && e == cudaSuccess; ++k) e = iteration();
        const cudaError_t e2 = cudaStreamEndCapture(cur, &graph);
        cur = s;
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&cache->exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        nl = nl0;  // nothing ran during the capture
        if (e != cudaSuccess) {
            cg_graph_release(*cache);
            return e;
        }
        for (int k = 0; k < 5; ++k) cache->key[k] = key[k];
        cache->launches = 9 * kChunk;
    }
    int64_t it = 0;
    double hs[4] = {0.0, 0.0, 0.0, 0.0};
    bool converged = false;
    if (cache && cache->exec) {
        while (it + kChunk <= max_iter) {
            if ((e = cudaGraphLaunch(cache->exec, s)) != cudaSuccess) break;
            nl += cache->launches;
            it += kChunk;
            if ((e = cudaMemcpyAsync(hs, sc, sizeof(hs), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
                break;
            if ((e = cudaStreamSynchronize(s)) != cudaSuccess) break;
            if (std::sqrt(hs[3]) <= tol * std::sqrt(2.0)) {
                converged = true;
                break;
            }
        }
    }
    for (; !converged && e == cudaSuccess && it < max_iter; ++it) {
        if ((e = iteration()) != cudaSuccess) break;
        if ((it & 7) == 7 || it + 1 == max_iter) {
            if ((e = cudaMemcpyAsync(hs, sc, sizeof(hs), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
                break;
            if ((e = cudaStreamSynchronize(s)) != cudaSuccess) break;
            if (std::sqrt(hs[3]) <= tol * std::sqrt(2.0)) {
                ++it;
                break;
            }
        }
    }
    double xu = 0.0, xv = 0.0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&xu, x + u, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&xv, x + v, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    *R_out = xu - xv;
    if (iters_out) *iters_out = it;
    if (launches) *launches += nl;
    return cudaGetLastError();
}

}  // namespace kc
