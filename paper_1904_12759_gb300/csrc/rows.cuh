// Row traversal for power-law graphs: rows with at most LONG_ROW entries are
// handled one thread per row; longer rows (hubs) are queued and handled one
// warp per row (lanes stride over the row, fixed shuffle tree), so a hub's
// latency-bound sequential loop never holds up a whole kernel.  Each row's
// result depends only on the row, not on the queue order.
#pragma once

#include "mcx_internal.cuh"

namespace mcx {

constexpr int64_t LONG_ROW = 32;

// Append the rows longer than LONG_ROW to queue (qn must start at 0).
__global__ void k_find_long_rows(int64_t n, const int64_t *__restrict__ rp, int32_t *__restrict__ queue,
                                 unsigned int *qn);

// y = s A x for rows of at most LONG_ROW entries, one thread per row (long rows
// are skipped).  s = *scale if scale is not NULL, else 1.  done: optional flag;
// when set the kernel returns at once.
__global__ void k_spmv_short(int64_t n, const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                             const double *__restrict__ val, const double *__restrict__ x, const double *scale,
                             double *__restrict__ y, const int32_t *done);

// y = s A x for the queued long rows, one warp per row.
__global__ void k_spmv_long(const int32_t *__restrict__ queue, const unsigned int *qn,
                            const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                            const double *__restrict__ val, const double *__restrict__ x, const double *scale,
                            double *__restrict__ y, const int32_t *done);

// y = A x over all rows; queue: int32 [n] scratch, qn: one counter (device).
cudaError_t spmv_hybrid(int64_t n, const int64_t *rp, const int32_t *col, const double *val, const double *x,
                        double *y, int32_t *queue, unsigned int *qn, cudaStream_t st);

}  // namespace mcx
