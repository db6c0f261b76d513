// Sparse products on the caller's CSR arrays: the hybrid SpMV of rows.cuh, and
// power iteration for lambda_max of a symmetric A >= 0 (Sec. 6 sets
// beta = 1/lambda_max; the paper notes finding it is costly for large
// networks, so it runs here on the GPU).
//
// Power iteration: x_0 = 1 with scale s_0 = 1/sqrt(n); iteration k computes
// y = A (s_k x_k) (x_k unnormalised, s_k = 1/||x_k||), the Rayleigh quotient
// lambda_k = (s_k x_k) . y and s_{k+1} = 1/||y||, then x_{k+1} = y (ping-pong
// buffers).  Per iteration: the short-row SpMV, the long-row SpMVs (hubs, one
// warp or one block per row; the long rows are listed once per call and their
// kernels launched only if the graph has such rows; without them the SpMV and
// the dot products run as one kernel), and a dot-product
// pass whose block partials the last block to finish reduces in a fixed order,
// so the result does not depend on scheduling.  Iterations stop when
// |lambda_k - lambda_{k-1}| <= tol |lambda_k|; the host checks every CHECK
// iterations and launches after convergence return at once.
#include <math.h>

#include <algorithm>

#include "rows.cuh"
#include "launch.h"

namespace mcx {

__global__ void k_find_long_rows(int64_t n, const int64_t *__restrict__ rp, int32_t *__restrict__ queue,
                                 unsigned int *qn) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t len = rp[i + 1] - rp[i];
        if (len > HUGE_ROW) queue[n - 1 - (int64_t)atomicAdd(qn + 1, 1u)] = (int32_t)i;
        else if (len > LONG_ROW) queue[atomicAdd(qn, 1u)] = (int32_t)i;
    }
}

__global__ void k_spmv_short(int64_t n, const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                             const double *__restrict__ val, const double *__restrict__ x, const double *scale,
                             double *__restrict__ y, const int32_t *done) {
    if (done && *(volatile const int32_t *)done) return;
    const double s = scale ? *scale : 1.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p0 = rp[i], p1 = rp[i + 1];
        if (p1 - p0 > LONG_ROW) continue;
        double acc = 0.0;
        for (int64_t p = p0; p < p1; ++p) acc = __fma_rn(val[p], x[col[p]], acc);
        y[i] = __dmul_rn(acc, s);
    }
}

__global__ void k_spmv_long(const int32_t *__restrict__ queue, const unsigned int *qn,
                            const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                            const double *__restrict__ val, const double *__restrict__ x, const double *scale,
                            double *__restrict__ y, const int32_t *done) {
    if (done && *(volatile const int32_t *)done) return;
    const double s = scale ? *scale : 1.0;
    const int lane = threadIdx.x & 31;
    const unsigned int nq = *qn;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; q < nq; q += warps) {
        const int32_t i = queue[q];
        double acc = 0.0;
        for (int64_t p = rp[i] + lane; p < rp[i + 1]; p += 32) acc = __fma_rn(val[p], x[col[p]], acc);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) y[i] = __dmul_rn(acc, s);
    }
}

__global__ void __launch_bounds__(ROW_BLOCK) k_spmv_huge(int64_t n, const int32_t *__restrict__ queue,
                                                         const unsigned int *qn, const int64_t *__restrict__ rp,
                                                         const int32_t *__restrict__ col,
                                                         const double *__restrict__ val,
                                                         const double *__restrict__ x, const double *scale,
                                                         double *__restrict__ y, const int32_t *done) {
    __shared__ double sh[ROW_BLOCK / 32];
    if (done && *(volatile const int32_t *)done) return;  // uniform over the grid
    const double s = scale ? *scale : 1.0;
    const unsigned int nq = qn[1];
    for (unsigned int b = blockIdx.x; b < nq; b += gridDim.x) {
        const int32_t i = queue[n - 1 - (int64_t)b];
        double acc = 0.0;
        for (int64_t p = rp[i] + threadIdx.x; p < rp[i + 1]; p += ROW_BLOCK) acc = __fma_rn(val[p], x[col[p]], acc);
        acc = block_sum_row(acc, sh);
        if (threadIdx.x == 0) y[i] = __dmul_rn(acc, s);
    }
}

cudaError_t spmv_hybrid(int64_t n, const int64_t *rp, const int32_t *col, const double *val, const double *x,
                        double *y, int32_t *queue, unsigned int *qn, cudaStream_t st) {
    const unsigned nb = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 32));
    cudaError_t e = cudaMemsetAsync(qn, 0, 2 * sizeof(unsigned int), st);
    if (e != cudaSuccess) return e;
    k_find_long_rows<<<nb, 256, 0, st>>>(n, rp, queue, qn);
    k_spmv_short<<<nb, 256, 0, st>>>(n, rp, col, val, x, nullptr, y, nullptr);
    k_spmv_long<<<152 * 8, 256, 0, st>>>(queue, qn, rp, col, val, x, nullptr, y, nullptr);
    k_spmv_huge<<<152 * 2, ROW_BLOCK, 0, st>>>(n, queue, qn, rp, col, val, x, nullptr, y, nullptr);
    return cudaGetLastError();
}

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
    uint32_t qn[2];  // long rows, huge rows
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
        s->qn[0] = 0;
        s->qn[1] = 0;
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

// The last block of a dot pass: the block partials in block order, then the
// Rayleigh quotient lambda = (s x) . y, the next scale 1/||y|| and the test.
__device__ __forceinline__ void power_finish(PowerScalars *sc, const double *part, double tol, double (*sh)[2]) {
    __threadfence();
    double a = 0.0, b = 0.0;
    for (int k = threadIdx.x; k < (int)gridDim.x; k += PI_THREADS) {
        a += ((volatile const double *)part)[2 * k];
        b += ((volatile const double *)part)[2 * k + 1];
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

// (s x) . y and y . y by blocks in a fixed grid-stride order; the last block
// reduces the block partials in block order and updates the scalars.
__global__ void __launch_bounds__(PI_THREADS) k_power_dots(int64_t n, const double *__restrict__ x,
                                                           const double *__restrict__ y, double *__restrict__ part,
                                                           PowerScalars *sc, double tol) {
    __shared__ double sh[PI_THREADS / 32][2];
    __shared__ bool last;
    if (*(volatile int32_t *)&sc->done) return;  // uniform over the grid
    const double s = sc->inv_norm;
    double xy = 0.0, yy = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * PI_THREADS + threadIdx.x; i < n; i += (int64_t)gridDim.x * PI_THREADS) {
        const double yi = y[i];
        xy = __fma_rn(__dmul_rn(s, x[i]), yi, xy);
        yy = __fma_rn(yi, yi, yy);
    }
    block_sum2(xy, yy, sh);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = xy;
        part[2 * blockIdx.x + 1] = yy;
        __threadfence();
        last = atomicAdd(&sc->ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last) power_finish(sc, part, tol, sh);
}

// One whole iteration for matrices without rows above LONG_ROW entries: y = A (s x)
// one thread per row, and the dot products x . y, y . y in the same pass (per-thread
// sums in grid-stride order, fixed block tree, the last block reduces the block
// partials in block order).  The grid must not exceed PI_MAX_BLOCKS blocks.
__global__ void __launch_bounds__(PI_THREADS) k_power_fused(int64_t n, const int64_t *__restrict__ rp,
                                                            const int32_t *__restrict__ col,
                                                            const double *__restrict__ val,
                                                            const double *__restrict__ x, double *__restrict__ y,
                                                            double *__restrict__ part, PowerScalars *sc,
                                                            double tol) {
    __shared__ double sh[PI_THREADS / 32][2];
    __shared__ bool last;
    if (*(volatile int32_t *)&sc->done) return;  // uniform over the grid
    const double s = sc->inv_norm;
    double xy = 0.0, yy = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * PI_THREADS + threadIdx.x; i < n; i += (int64_t)gridDim.x * PI_THREADS) {
        double acc = 0.0;
        for (int64_t p = rp[i]; p < rp[i + 1]; ++p) acc = __fma_rn(val[p], x[col[p]], acc);
        const double yi = __dmul_rn(acc, s);
        y[i] = yi;
        xy = __fma_rn(__dmul_rn(s, x[i]), yi, xy);
        yy = __fma_rn(yi, yi, yy);
    }
    block_sum2(xy, yy, sh);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = xy;
        part[2 * blockIdx.x + 1] = yy;
        __threadfence();
        last = atomicAdd(&sc->ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last) power_finish(sc, part, tol, sh);
}

}  // namespace

cudaError_t run_power_iteration(int64_t n, const int64_t *row_ptr, const int32_t *col, const double *val,
                                int32_t max_iters, double tol, double *work, double *lambda, int32_t *iters,
                                cudaStream_t st) {
    double *buf[2] = {work, work + n};
    double *part = work + 2 * n;
    PowerScalars *s = reinterpret_cast<PowerScalars *>(work + 2 * n + 2 * PI_MAX_BLOCKS);
    int32_t *queue = reinterpret_cast<int32_t *>(work + 2 * n + 2 * PI_MAX_BLOCKS + 8);
    const int64_t want = (n + PI_THREADS - 1) / PI_THREADS;
    const int nb = (int)std::max<int64_t>(1, std::min<int64_t>(PI_MAX_BLOCKS, want));
    const unsigned nrow = (unsigned)std::max<int64_t>(1, std::min<int64_t>(want, 152 * 32));
    k_init<<<nb, PI_THREADS, 0, st>>>(n, buf[0], s);
    k_find_long_rows<<<nrow, 256, 0, st>>>(n, row_ptr, queue, s->qn);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    PowerScalars hs{};
    // the queue sizes decide which row kernels each iteration needs
    if ((e = cudaMemcpyAsync(&hs, s, sizeof(hs), cudaMemcpyDeviceToHost, st)) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
    const bool any_long = hs.qn[0] > 0, any_huge = hs.qn[1] > 0;
    int32_t launched = 0;
    while (launched < max_iters) {
        const int32_t batch = std::min<int32_t>(CHECK, max_iters - launched);
        for (int32_t b = 0; b < batch; ++b, ++launched) {
            const double *x = buf[launched & 1];
            double *y = buf[(launched + 1) & 1];
            if (!any_long && !any_huge) {
                k_power_fused<<<nb, PI_THREADS, 0, st>>>(n, row_ptr, col, val, x, y, part, s, tol);
                continue;
            }
            k_spmv_short<<<nrow, 256, 0, st>>>(n, row_ptr, col, val, x, &s->inv_norm, y, &s->done);
            if (any_long)
                k_spmv_long<<<152 * 8, 256, 0, st>>>(queue, s->qn, row_ptr, col, val, x, &s->inv_norm, y, &s->done);
            if (any_huge)
                k_spmv_huge<<<152 * 2, ROW_BLOCK, 0, st>>>(n, queue, s->qn, row_ptr, col, val, x, &s->inv_norm, y,
                                                          &s->done);
            k_power_dots<<<nb, PI_THREADS, 0, st>>>(n, x, y, part, s, tol);
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
