// Row traversal for power-law graphs: rows with at most LONG_ROW entries are
// handled one thread per row; longer rows (hubs) are queued once per call and
// handled one warp per row, and rows above HUGE_ROW entries one block of
// ROW_BLOCK threads per row (lanes stride over the row, fixed reduction trees),
// so no hub's sequential loop holds up a whole kernel.  Each row's result
// depends only on the row, not on the queue order.
#pragma once

#include "mcx_internal.cuh"

namespace mcx {

constexpr int64_t LONG_ROW = 32;
constexpr int64_t HUGE_ROW = 1024;
constexpr int ROW_BLOCK = 256;

// Queue the rows longer than LONG_ROW: rows of at most HUGE_ROW entries at
// queue[0, qn[0]), longer ones at queue[n - qn[1], n) (filled from the back).
// qn[0] and qn[1] must start at 0.
__global__ void k_find_long_rows(int64_t n, const int64_t *__restrict__ rp, int32_t *__restrict__ queue,
                                 unsigned int *qn);

// y = s A x for rows of at most LONG_ROW entries, one thread per row (long rows
// are skipped).  s = *scale if scale is not NULL, else 1.  done: optional flag;
// when set the kernel returns at once.
__global__ void k_spmv_short(int64_t n, const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                             const double *__restrict__ val, const double *__restrict__ x, const double *scale,
                             double *__restrict__ y, const int32_t *done);

// y = s A x for the queued rows of LONG_ROW..HUGE_ROW entries, one warp per row.
__global__ void k_spmv_long(const int32_t *__restrict__ queue, const unsigned int *qn,
                            const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                            const double *__restrict__ val, const double *__restrict__ x, const double *scale,
                            double *__restrict__ y, const int32_t *done);

// y = s A x for the queued rows above HUGE_ROW entries, one block per row.
__global__ void k_spmv_huge(int64_t n, const int32_t *__restrict__ queue, const unsigned int *qn,
                            const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                            const double *__restrict__ val, const double *__restrict__ x, const double *scale,
                            double *__restrict__ y, const int32_t *done);

// Fixed-shape FP64 sum over a block of ROW_BLOCK threads; the result is valid
// in thread 0.  sh: ROW_BLOCK / 32 doubles of shared memory.
__device__ __forceinline__ double block_sum_row(double v, double *sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double r = 0.0;
    if (warp == 0) {
        r = lane < ROW_BLOCK / 32 ? sh[lane] : 0.0;
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
    }
    __syncthreads();  // sh reusable
    return r;
}

// y = A x over all rows (short, long and huge kernels); queue: int32 [n]
// scratch, qn: two counters (device).
cudaError_t spmv_hybrid(int64_t n, const int64_t *rp, const int32_t *col, const double *val, const double *x,
                        double *y, int32_t *queue, unsigned int *qn, cudaStream_t st);

}  // namespace mcx
