// Power iteration for lambda_max of a symmetric A >= 0 (Sec. 6 sets
// beta = 1/lambda_max; the paper notes finding it is costly for large
// networks, so it runs here on the GPU over the caller's CSR arrays).
//
// Iteration: y = A x (one thread per row, grid-stride), block partial sums of
// x.y and y.y written per block; one block then sums the partials in block
// order (deterministic), forms the Rayleigh quotient lambda = x.y (x has unit
// norm), tests |lambda - lambda_prev| <= tol |lambda| and sets x = y/||y||.
// The host checks the converged flag every CHECK iterations.
#include <math.h>

#include <algorithm>

#include "mcx_internal.cuh"

namespace mcx {
namespace {

constexpr int SPMV_THREADS = 256;
constexpr int SPMV_MAX_BLOCKS = 1024;
constexpr int CHECK = 16;

struct PowerScalars {
    double lambda;
    double lambda_prev;
    double inv_norm;
    int32_t done;
    int32_t iters;
};

__global__ void k_init(int64_t n, double *x, PowerScalars *s) {
    const double v = 1.0 / sqrt((double)n);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] = v;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        s->lambda = 0.0;
        s->lambda_prev = 0.0;
        s->inv_norm = 0.0;
        s->done = 0;
        s->iters = 0;
    }
}

__device__ __forceinline__ double block_sum(double v, double *sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r += sh[w];
    return r;  // valid in thread 0
}

__global__ void __launch_bounds__(SPMV_THREADS) k_spmv(int64_t n, const int64_t *__restrict__ rp,
                                                       const int32_t *__restrict__ col,
                                                       const double *__restrict__ val, const double *__restrict__ x,
                                                       double *__restrict__ y, double *__restrict__ part,
                                                       const PowerScalars *s) {
    __shared__ double sh[SPMV_THREADS / 32];
    if (s->done) return;
    double xy = 0.0, yy = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int64_t p = rp[i]; p < rp[i + 1]; ++p) acc += val[p] * x[col[p]];
        y[i] = acc;
        xy += x[i] * acc;
        yy += acc * acc;
    }
    const double a = block_sum(xy, sh);
    const double b = block_sum(yy, sh);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = a;
        part[2 * blockIdx.x + 1] = b;
    }
}

__global__ void k_finish(int nblocks, const double *__restrict__ part, double tol, PowerScalars *s) {
    if (s->done) return;
    double xy = 0.0, yy = 0.0;
    for (int b = 0; b < nblocks; ++b) {
        xy += part[2 * b];
        yy += part[2 * b + 1];
    }
    s->lambda_prev = s->lambda;
    s->lambda = xy;
    s->iters += 1;
    s->inv_norm = yy > 0.0 ? 1.0 / sqrt(yy) : 0.0;
    if (yy == 0.0 || (s->iters > 1 && fabs(xy - s->lambda_prev) <= tol * fabs(xy))) s->done = 1;
}

__global__ void k_scale(int64_t n, const double *__restrict__ y, double *__restrict__ x, const PowerScalars *s) {
    if (s->done) return;
    const double c = s->inv_norm;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] = y[i] * c;
}

}  // namespace

cudaError_t run_power_iteration(int64_t n, const int64_t *row_ptr, const int32_t *col, const double *val,
                                int32_t max_iters, double tol, double *work, double *lambda, int32_t *iters,
                                cudaStream_t st) {
    double *x = work, *y = work + n, *part = work + 2 * n;
    PowerScalars *s = reinterpret_cast<PowerScalars *>(work + 2 * n + 2 * SPMV_MAX_BLOCKS);
    const int nb = (int)std::min<int64_t>(SPMV_MAX_BLOCKS, (n + SPMV_THREADS - 1) / SPMV_THREADS);
    k_init<<<nb, SPMV_THREADS, 0, st>>>(n, x, s);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    PowerScalars hs{};
    for (int32_t it = 0; it < max_iters; it += CHECK) {
        const int32_t batch = std::min<int32_t>(CHECK, max_iters - it);
        for (int32_t b = 0; b < batch; ++b) {
            k_spmv<<<nb, SPMV_THREADS, 0, st>>>(n, row_ptr, col, val, x, y, part, s);
            k_finish<<<1, 1, 0, st>>>(nb, part, tol, s);
            k_scale<<<nb, SPMV_THREADS, 0, st>>>(n, y, x, s);
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if ((e = cudaMemcpyAsync(&hs, s, sizeof(hs), cudaMemcpyDeviceToHost, st)) != cudaSuccess) return e;
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
        if (hs.done) break;
    }
    if (lambda) *lambda = hs.lambda;
    if (iters) *iters = hs.iters;
    return cudaSuccess;
}

}  // namespace mcx
