// Host-side launch helpers of the mcx library, declared for the .cu files that
// define and call them (plain host code: kernels never see these).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include "mcx_internal.cuh"

namespace mcx {

// NVTX range over one C-ABI call (host side: its validation and the work it
// enqueues), named after the call; free when no profiler is attached.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

cudaError_t launch_prep(mcx_plan *plan, const int64_t *row_ptr, const int32_t *col, const double *val,
                        cudaStream_t st, uint32_t *host_status);
cudaError_t launch_export(const mcx_plan *plan, int32_t *deg, int64_t *row_start, uint8_t *weighted, float *ir32,
                          float *d32, double *ir64, double *d64, int32_t *ecol, int32_t *acol, uint32_t *thr,
                          cudaStream_t st);
cudaError_t launch_pack_v(mcx_plan *plan, const double *v, cudaStream_t st);

struct EstimateArgs {
    const int32_t *entries;
    int64_t n_entries;
    uint64_t paths;
    double t;
    int mode;
    int nsteps;
    int precision;
    uint64_t seed;
    uint64_t path_offset;
    double *mean;
    double *sem;
};
cudaError_t launch_estimate(mcx_plan *plan, const EstimateArgs &a, cudaStream_t st);
struct RqmcArgs {
    const int32_t *entries;
    int64_t n_entries;
    uint32_t log2q;
    uint32_t replicates;
    uint32_t r0;  // first replicate index
    double t;
    int mode;
    int nsteps;
    int precision;
    uint64_t seed;
    double *mean;
    double *sem;
};
// Multilevel level difference N vs N/2 (v already packed into the node records).
cudaError_t launch_level_difference(mcx_plan *plan, const EstimateArgs &a, cudaStream_t st);
// Randomised-QMC estimate (v already packed into the node records).
cudaError_t launch_estimate_rqmc(mcx_plan *plan, const RqmcArgs &a, cudaStream_t st);
cudaError_t launch_estimate_noalloc(mcx_plan *plan, const double *v, const EstimateArgs &a, cudaStream_t st,
                                    bool *too_large);
uint64_t noalloc_max_partials();
cudaError_t launch_estimate_forward(mcx_plan *plan, const double *v, double t, int mode, int nsteps, uint64_t paths,
                                    uint64_t seed, uint64_t path_offset, int precision, double *x, double *sem,
                                    cudaStream_t st);
// Stream-ordered allocation from the library's memory pool of the current
// device (created on first use; memory freed to it stays reserved for the next
// plan instead of being released to the system, so plans are created and destroyed
// without device-wide synchronisation).
cudaError_t pool_alloc(void **p, size_t bytes, cudaStream_t st);
void pool_free(void *p, cudaStream_t st);
// Device allocations outside the pool (grow-only scratch, batch and network
// arrays).  Like pool_alloc they honour the failure-injection test hook
// (mcx_debug_fail_alloc): the armed allocation returns cudaErrorMemoryAllocation.
cudaError_t dev_malloc(void **p, size_t bytes);
template <typename T>
inline cudaError_t dev_malloc(T **p, size_t bytes) {
    return dev_malloc(reinterpret_cast<void **>(p), bytes);
}
void dev_free(void *p);
cudaError_t launch_total_communicability(mcx_plan *plan, double t, int mode, int nsteps, uint64_t paths,
                                         uint64_t seed, uint64_t path_offset, int precision, double *tc, double *sem,
                                         cudaStream_t st);
cudaError_t launch_trace_forward(mcx_plan *plan, const double *v, double t, int mode, int nsteps, uint64_t seed,
                                 uint64_t first_path, uint32_t count, int precision, int32_t *start, int32_t *end,
                                 uint32_t *njumps, uint64_t *hash, double *logw, cudaStream_t st);
cudaError_t launch_trace(mcx_plan *plan, double t, int mode, int nsteps, int32_t entry, uint64_t seed,
                         uint64_t first_path, uint32_t count, int precision, int32_t *end, uint32_t *njumps,
                         uint64_t *hash, double *logw, cudaStream_t st);
// The batched control variate's pre-pass over the rows of its slot CSR (cv.cu):
// t_row gives each row its own horizon and t3inv_row the FP64 1/(t*t*t) of it,
// so that the rows of many problems are prepared at once.  The batched form
// builds its row schedule and sliced ELL copy once, then per run calls
// cv_taylor_rows without the third Taylor term and cv_cubic_rows, which forms
// A^3 v and A c3 in one pass; both give the bits of mcx_cv_prepare and
// mcx_cv_coefficients on each problem alone.
// Row schedule of the control variate's row passes (cv.cu): order [n] int32,
// cnt [CV_ROW_CNT] and hist [ceil(n / CV_ROW_WINDOW) + 1] uint32, device memory.
constexpr int CV_ROW_CNT = 8;
constexpr int CV_ROW_WINDOW = 256;
struct CvRowSchedule {
    int32_t *order;
    uint32_t *cnt;
    uint32_t *hist;
};
// Sliced ELL copy of a schedule's short rows: chunk k holds the short rows
// 32k .. 32k + 31 of the schedule, entry e of the chunk's row l at
// chunk[k] + 32 e + l of col / val; len [short rows] their lengths.
struct CvSell {
    const int32_t *col;
    const double *val;
    const int64_t *chunk;
    const uint8_t *len;
};
cudaError_t cv_taylor_rows(int64_t n, const int64_t *row_ptr, const int32_t *col, const double *val,
                           const double *v, double t, const double *t_row, const CvRowSchedule &s, const CvSell *ell,
                           double2 *g, double *lam, double *taylor, float *features, bool third, cudaStream_t st);
cudaError_t cv_cubic_rows(int64_t n, const int64_t *row_ptr, const int32_t *col, const double *val,
                          const double *taylor, const float *y, const double *t_row, const double *t3inv_row,
                          const CvRowSchedule &s, const CvSell *ell, double2 *q, double2 *ab, double *h,
                          cudaStream_t st);
cudaError_t run_power_iteration(int64_t n, const int64_t *row_ptr, const int32_t *col, const double *val,
                                int32_t max_iters, double tol, double *work, double *lambda, int32_t *iters,
                                cudaStream_t st);

}  // namespace mcx
