// Power iteration for lambda_max of a symmetric A >= 0 (Sec. 6 sets
// beta = 1/lambda_max; the paper notes finding it is costly for large
// networks, so it runs here on the GPU over the caller's CSR arrays).
//
// x_0 = 1 with scale s_0 = 1/sqrt(n); iteration k computes y = A (s_k x_k)
// (x_k unnormalised, s_k = 1/||x_k||), the Rayleigh quotient
// lambda_k = (s_k x_k) . y and s_{k+1} = 1/||y||, then x_{k+1} = y: one
// fused kernel per iteration, ping-pong buffers, no separate scaling pass.
// One thread per row, so each stored entry costs one FP64 fma slot.
// Each block writes its two partial dot products; the last block to finish
// (atomic ticket after a fence) reduces all partials in a fixed tree order,
// so the result does not depend on block scheduling.  Iterations stop when
// |lambda_k - lambda_{k-1}| <= tol |lambda_k|; the host checks every CHECK
// launches and launches after convergence return at once.
#include <math.h>

#include <algorithm>

#include "mcx_internal.cuh"

namespace mcx {
namespace {

constexpr int PI_THREADS = 256;
constexpr int PI_MAX_BLOCKS = 1024;
constexpr int CHECK = 8;

struct PowerScalars {
    double lambda;
    double lambda_prev;
    double inv_norm;
    int32_t done;
    int32_t iters;
    uint32_t ticket;
    uint32_t pad;
};

__global__ void k_init(int64_t n, double *x, PowerScalars *s) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] = 1.0;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        s->lambda = 0.0;
        s->lambda_prev = 0.0;
        s->inv_norm = 1.0 / sqrt((double)n);
        s->done = 0;
        s->iters = 0;
        s->ticket = 0;
    }
}

// Fixed-shape block reduction of (a, b); result valid in thread 0.
__device__ __forceinline__ void block_sum2(double &a, double &b, double (*sh)[2]) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        sh[warp][0] = a;
        sh[warp][1] = b;
    }
    __syncthreads();
    if (warp == 0) {
        a = lane < PI_THREADS / 32 ? sh[lane][0] : 0.0;
        b = lane < PI_THREADS / 32 ? sh[lane][1] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, o);
            b += __shfl_xor_sync(0xffffffffu, b, o);
        }
    }
}

__global__ void __launch_bounds__(PI_THREADS) k_power_step(int64_t n, const int64_t *__restrict__ rp,
                                                           const int32_t *__restrict__ col,
                                                           const double *__restrict__ val,
                                                           const double *__restrict__ x, double *__restrict__ y,
                                                           double *__restrict__ part, PowerScalars *sc, double tol) {
    __shared__ double sh[PI_THREADS / 32][2];
    __shared__ bool last;
    if (*(volatile int32_t *)&sc->done) return;  // uniform over the grid
    const double s = sc->inv_norm;
    // one thread per row: each stored entry costs exactly one FP64 fma slot (the
    // FP64 pipe, not memory, bounds this kernel on this GPU)
    double xy = 0.0, yy = 0.0;
    for (int64_t row = (int64_t)blockIdx.x * PI_THREADS + threadIdx.x; row < n; row += (int64_t)gridDim.x * PI_THREADS) {
        double acc = 0.0;
        const int64_t p1 = rp[row + 1];
        for (int64_t p = rp[row]; p < p1; ++p) acc = __fma_rn(val[p], x[col[p]], acc);
        acc = __dmul_rn(acc, s);
        y[row] = acc;
        xy = __fma_rn(__dmul_rn(s, x[row]), acc, xy);
        yy = __fma_rn(acc, acc, yy);
    }
    block_sum2(xy, yy, sh);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = xy;
        part[2 * blockIdx.x + 1] = yy;
        __threadfence();
        last = atomicAdd(&sc->ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    // last block: fixed-order reduction of all block partials
    __threadfence();
    double a = 0.0, b = 0.0;
    for (int k = threadIdx.x; k < (int)gridDim.x; k += PI_THREADS) {
        a += ((volatile double *)part)[2 * k];
        b += ((volatile double *)part)[2 * k + 1];
    }
    __syncthreads();
    block_sum2(a, b, sh);
    if (threadIdx.x == 0) {
        const int32_t it = sc->iters + 1;
        sc->lambda_prev = sc->lambda;
        sc->lambda = a;
        sc->iters = it;
        sc->inv_norm = b > 0.0 ? 1.0 / sqrt(b) : 0.0;
        sc->ticket = 0;
        if (b == 0.0 || (it > 1 && fabs(a - sc->lambda_prev) <= tol * fabs(a))) sc->done = 1;
    }
}

}  // namespace

cudaError_t run_power_iteration(int64_t n, const int64_t *row_ptr, const int32_t *col, const double *val,
                                int32_t max_iters, double tol, double *work, double *lambda, int32_t *iters,
                                cudaStream_t st) {
    double *buf[2] = {work, work + n};
    double *part = work + 2 * n;
    PowerScalars *s = reinterpret_cast<PowerScalars *>(work + 2 * n + 2 * PI_MAX_BLOCKS);
    const int64_t want = (n + PI_THREADS - 1) / PI_THREADS;
    const int nb = (int)std::max<int64_t>(1, std::min<int64_t>(PI_MAX_BLOCKS, want));
    k_init<<<nb, PI_THREADS, 0, st>>>(n, buf[0], s);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    PowerScalars hs{};
    int32_t launched = 0;
    while (launched < max_iters) {
        const int32_t batch = std::min<int32_t>(CHECK, max_iters - launched);
        for (int32_t b = 0; b < batch; ++b, ++launched)
            k_power_step<<<nb, PI_THREADS, 0, st>>>(n, row_ptr, col, val, buf[launched & 1], buf[(launched + 1) & 1],
                                                    part, s, tol);
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
