// C-ABI entry points (include/mcx.h): argument checks, plan ownership and
// status handling around the kernels of prep.cu, walk.cu and spmv.cu.
#include <math.h>
#include <stdlib.h>

#include <atomic>
#include <mutex>
#include <new>

#include "mcx_internal.cuh"
#include "launch.h"

using namespace mcx;

namespace {

mcx_status from_cuda(cudaError_t e) {
    if (e == cudaSuccess) return MCX_OK;
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();  // clear the sticky-free allocation error
        return MCX_E_OOM;
    }
    return MCX_E_CUDA;
}

// The plan's own arrays come from the memory pool; its grow-only scratch from cudaMalloc.
// Called with no work of the plan in flight.
void free_plan(mcx_plan *p) {
    if (!p) return;
    pool_free(p->node, 0);
    pool_free(p->node64, 0);
    pool_free(p->edge_col, 0);
    pool_free(p->edge16, 0);
    pool_free(p->status, 0);
    dev_free(p->scratch);
    dev_free(p->fwd);
    delete p;
}

std::mutex g_pool_mu;
cudaMemPool_t g_pools[64];
bool g_pool_ready[64] = {};

// Failure injection (test hook): g_fail_in > 0 counts down the device
// allocations still to succeed before one fails; 0 is disarmed.
std::atomic<int64_t> g_fail_in{0};
std::atomic<int64_t> g_allocs{0};

bool injected_failure() {
    g_allocs.fetch_add(1);
    int64_t c = g_fail_in.load();
    while (c > 0) {
        if (g_fail_in.compare_exchange_weak(c, c - 1)) return c == 1;
    }
    return false;
}

}  // namespace

namespace mcx {

cudaError_t dev_malloc(void **p, size_t bytes) {
    *p = nullptr;
    if (injected_failure()) return cudaErrorMemoryAllocation;
    return cudaMalloc(p, bytes ? bytes : 1);
}

void dev_free(void *p) {
    if (p) cudaFree(p);
}

cudaError_t pool_alloc(void **p, size_t bytes, cudaStream_t st) {
    *p = nullptr;
    if (injected_failure()) return cudaErrorMemoryAllocation;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    cudaMemPool_t pool;
    {
        std::lock_guard<std::mutex> lock(g_pool_mu);
        if (!g_pool_ready[dev]) {
            cudaMemPoolProps props{};
            props.allocType = cudaMemAllocationTypePinned;
            props.location.type = cudaMemLocationTypeDevice;
            props.location.id = dev;
            if ((e = cudaMemPoolCreate(&g_pools[dev], &props)) != cudaSuccess) return e;
            uint64_t keep = ~0ull;  // never trim: freed blocks serve the next plan
            cudaMemPoolSetAttribute(g_pools[dev], cudaMemPoolAttrReleaseThreshold, &keep);
            g_pool_ready[dev] = true;
        }
        pool = g_pools[dev];
    }
    return cudaMallocFromPoolAsync(p, bytes ? bytes : 1, pool, st);
}

void pool_free(void *p, cudaStream_t st) {
    if (p) cudaFreeAsync(p, st);
}

}  // namespace mcx

extern "C" {

int mcx_version(void) { return 100; }

int64_t mcx_debug_fail_alloc(int64_t k) {
    g_fail_in.store(k > 0 ? k : 0);
    return g_allocs.load();
}

mcx_status mcx_debug_pool_usage(uint64_t *used, uint64_t *reserved) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return MCX_E_CUDA;
    cudaMemPool_t pool;
    {
        std::lock_guard<std::mutex> lock(g_pool_mu);
        if (!g_pool_ready[dev]) {
            if (used) *used = 0;
            if (reserved) *reserved = 0;
            return MCX_OK;
        }
        pool = g_pools[dev];
    }
    unsigned long long u = 0, r = 0;
    if (cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &u) != cudaSuccess ||
        cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &r) != cudaSuccess)
        return MCX_E_CUDA;
    if (used) *used = (uint64_t)u;
    if (reserved) *reserved = (uint64_t)r;
    return MCX_OK;
}

const char *mcx_status_string(int s) {
    switch (s) {
        case MCX_OK: return "ok";
        case MCX_E_INVALID: return "invalid argument or malformed CSR";
        case MCX_E_NEG_OFFDIAG: return "negative off-diagonal entry: -L is not a generator";
        case MCX_E_NONFINITE: return "non-finite value in A or v";
        case MCX_E_NEG_V: return "forward form needs v >= 0 with a positive sum";
        case MCX_E_CUDA: return "CUDA runtime error";
        case MCX_E_OOM: return "device allocation failed";
        case MCX_E_TIMEOUT: return "bounded device wait gave up";
        case MCX_E_UNSUPPORTED: return "unsupported request";
        case MCX_E_OVERFLOW: return "estimate overflowed FP64";
        default: return "unknown status";
    }
}

mcx_status mcx_plan_create(int64_t n, int64_t nnz, const int64_t *row_ptr, const int32_t *col, const double *val,
                           uint32_t flags, void *stream, mcx_plan **out) {
    NvtxRange nvtx("mcx_plan_create");
    if (!out) return MCX_E_INVALID;
    *out = nullptr;
    if (n < 0 || n >= (int64_t)0x7fffffff || nnz < 0 || !row_ptr || (nnz > 0 && (!col || !val)))
        return MCX_E_INVALID;
    if (flags & ~MCX_PLAN_HOST_INPUT) return MCX_E_INVALID;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    mcx_plan *p = new (std::nothrow) mcx_plan();
    if (!p) return MCX_E_OOM;
    p->n = n;
    p->nnz = nnz;
    cudaGetDevice(&p->device);
    int64_t *d_rp = nullptr;
    int32_t *d_col = nullptr;
    double *d_val = nullptr;
    const bool host = (flags & MCX_PLAN_HOST_INPUT) != 0;
    mcx_status rc = MCX_OK;
    uint32_t dev_status = 0;
    do {
        cudaError_t e;
        const size_t nn = (size_t)(n > 0 ? n : 1);
        if ((e = pool_alloc(reinterpret_cast<void **>(&p->node), sizeof(NodeRec) * nn, st)) != cudaSuccess) { rc = from_cuda(e); break; }
        if ((e = pool_alloc(reinterpret_cast<void **>(&p->node64), sizeof(NodeRec64) * nn, st)) != cudaSuccess) { rc = from_cuda(e); break; }
        if ((e = pool_alloc(reinterpret_cast<void **>(&p->status), 4 * STATUS_WORDS, st)) != cudaSuccess) { rc = from_cuda(e); break; }
        if ((e = cudaMemsetAsync(p->status, 0, 4 * STATUS_WORDS, st)) != cudaSuccess) { rc = from_cuda(e); break; }
        p->device_bytes = (int64_t)((sizeof(NodeRec) + sizeof(NodeRec64)) * nn + 16);
        const int64_t *rp = row_ptr;
        const int32_t *cc = col;
        const double *vv = val;
        if (host) {
            if ((e = pool_alloc(reinterpret_cast<void **>(&d_rp), sizeof(int64_t) * (size_t)(n + 1), st)) != cudaSuccess) { rc = from_cuda(e); break; }
            if ((e = pool_alloc(reinterpret_cast<void **>(&d_col), sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1), st)) != cudaSuccess) { rc = from_cuda(e); break; }
            if ((e = pool_alloc(reinterpret_cast<void **>(&d_val), sizeof(double) * (size_t)(nnz > 0 ? nnz : 1), st)) != cudaSuccess) { rc = from_cuda(e); break; }
            if ((e = cudaMemcpyAsync(d_rp, row_ptr, sizeof(int64_t) * (size_t)(n + 1), cudaMemcpyHostToDevice, st)) != cudaSuccess) { rc = from_cuda(e); break; }
            if (nnz > 0) {
                if ((e = cudaMemcpyAsync(d_col, col, sizeof(int32_t) * (size_t)nnz, cudaMemcpyHostToDevice, st)) != cudaSuccess) { rc = from_cuda(e); break; }
                if ((e = cudaMemcpyAsync(d_val, val, sizeof(double) * (size_t)nnz, cudaMemcpyHostToDevice, st)) != cudaSuccess) { rc = from_cuda(e); break; }
            }
            rp = d_rp; cc = d_col; vv = d_val;
        }
        if ((e = launch_prep(p, rp, cc, vv, st, &dev_status)) != cudaSuccess) { rc = from_cuda(e); break; }
        if (dev_status & ST_BAD_STRUCT) rc = MCX_E_INVALID;
        else if (dev_status & ST_NONFINITE) rc = MCX_E_NONFINITE;
        else if (dev_status & ST_NEG_OFFDIAG) rc = MCX_E_NEG_OFFDIAG;
    } while (0);
    if (host) {  // stream-ordered: freed after the preparation that reads them
        pool_free(d_rp, st);
        pool_free(d_col, st);
        pool_free(d_val, st);
    }
    if (rc != MCX_OK) {
        cudaStreamSynchronize(st);
        free_plan(p);
        return rc;
    }
    *out = p;
    return MCX_OK;
}

mcx_status mcx_plan_get_info(const mcx_plan *p, mcx_plan_info *info) {
    if (!p || !info) return MCX_E_INVALID;
    info->n = p->n;
    info->nnz = p->nnz;
    info->nnz_off = p->nnz_off;
    info->weighted_rows = p->weighted_rows;
    info->max_deg = p->max_deg;
    info->reserved = 0;
    info->device_bytes = p->device_bytes + (int64_t)p->scratch_bytes + (int64_t)p->fwd_bytes;
    return MCX_OK;
}

static mcx_status check_common(const mcx_plan *p, double t, int functional, int32_t nsteps, int precision) {
    if (!p) return MCX_E_INVALID;
    if (!(t >= 0.0) || !isfinite(t)) return MCX_E_INVALID;
    if (functional != MCX_EXACT && functional != MCX_STRANG && functional != MCX_LIE) return MCX_E_INVALID;
    if (functional != MCX_EXACT && (nsteps < 1 || nsteps > (1 << 24))) return MCX_E_INVALID;
    if (precision != MCX_FP32 && precision != MCX_FP64) return MCX_E_INVALID;
    return MCX_OK;
}

mcx_status mcx_estimate(mcx_plan *p, const double *v, double t, int functional, int32_t nsteps,
                        uint64_t paths_per_entry, const int32_t *entries, int64_t n_entries, uint64_t seed,
                        uint64_t path_offset, int precision, double *mean, double *sem, void *stream) {
    NvtxRange nvtx("mcx_estimate");
    mcx_status rc = check_common(p, t, functional, nsteps, precision);
    if (rc != MCX_OK) return rc;
    if (n_entries == 0) return MCX_OK;  // nothing requested (an empty entry list may be NULL)
    if (!v || n_entries < 0 || paths_per_entry < 1 || !mean) return MCX_E_INVALID;
    if (!entries && n_entries != p->n) return MCX_E_INVALID;
    if (paths_per_entry > (1ull << 53)) return MCX_E_INVALID;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = launch_pack_v(p, v, st);
    if (e != cudaSuccess) return from_cuda(e);
    EstimateArgs a{};
    a.entries = entries;
    a.n_entries = n_entries;
    a.paths = paths_per_entry;
    a.t = t;
    a.mode = functional;
    a.nsteps = nsteps;
    a.precision = precision;
    a.seed = seed;
    a.path_offset = path_offset;
    a.mean = mean;
    a.sem = sem;
    return from_cuda(launch_estimate(p, a, st));
}

mcx_status mcx_estimate_level_difference(mcx_plan *p, const double *v, double t, int functional, int32_t nsteps,
                                         uint64_t paths_per_entry, const int32_t *entries, int64_t n_entries,
                                         uint64_t seed, uint64_t path_offset, int precision, double *mean,
                                         double *sem, void *stream) {
    NvtxRange nvtx("mcx_estimate_level_difference");
    mcx_status rc = check_common(p, t, functional, nsteps, precision);
    if (rc != MCX_OK) return rc;
    if (functional != MCX_STRANG && functional != MCX_LIE) return MCX_E_INVALID;
    if (nsteps < 2 || (nsteps & 1)) return MCX_E_INVALID;
    if (n_entries == 0) return MCX_OK;
    if (!v || n_entries < 0 || paths_per_entry < 1 || !mean) return MCX_E_INVALID;
    if (!entries && n_entries != p->n) return MCX_E_INVALID;
    if (paths_per_entry > (1ull << 53)) return MCX_E_INVALID;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = launch_pack_v(p, v, st);
    if (e != cudaSuccess) return from_cuda(e);
    EstimateArgs a{};
    a.entries = entries;
    a.n_entries = n_entries;
    a.paths = paths_per_entry;
    a.t = t;
    a.mode = functional;
    a.nsteps = nsteps;
    a.precision = precision;
    a.seed = seed;
    a.path_offset = path_offset;
    a.mean = mean;
    a.sem = sem;
    if (t == 0.0) {  // both functionals are 0: every difference is 0
        e = cudaMemsetAsync(mean, 0, sizeof(double) * (size_t)n_entries, st);
        if (e == cudaSuccess && sem) e = cudaMemsetAsync(sem, 0, sizeof(double) * (size_t)n_entries, st);
        return from_cuda(e);
    }
    return from_cuda(launch_level_difference(p, a, st));
}

mcx_status mcx_estimate_rqmc(mcx_plan *p, const double *v, double t, int functional, int32_t nsteps,
                             uint32_t log2_points, uint32_t replicates, uint32_t replicate_offset,
                             const int32_t *entries, int64_t n_entries, uint64_t seed, int precision, double *mean,
                             double *sem, void *stream) {
    NvtxRange nvtx("mcx_estimate_rqmc");
    mcx_status rc = check_common(p, t, functional, nsteps, precision);
    if (rc != MCX_OK) return rc;
    if (n_entries == 0) return MCX_OK;
    if (!v || n_entries < 0 || !mean || replicates < 1 || replicates > (1u << 16) || log2_points > MCX_QMC_MAX_LOG2)
        return MCX_E_INVALID;
    if (!entries && n_entries != p->n) return MCX_E_INVALID;
    if (((uint64_t)replicates << log2_points) > (1ull << 40)) return MCX_E_INVALID;
    if ((uint64_t)replicate_offset + replicates > 0xFFFFFFFFull) return MCX_E_INVALID;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = launch_pack_v(p, v, st);
    if (e != cudaSuccess) return from_cuda(e);
    if (t == 0.0) {  // exp(0 A) v = v: the plain estimator's copy path
        EstimateArgs a{};
        a.entries = entries;
        a.n_entries = n_entries;
        a.paths = 1;
        a.t = 0.0;
        a.mode = functional;
        a.nsteps = nsteps;
        a.precision = precision;
        a.mean = mean;
        a.sem = sem;
        return from_cuda(launch_estimate(p, a, st));
    }
    RqmcArgs a{};
    a.entries = entries;
    a.n_entries = n_entries;
    a.log2q = log2_points;
    a.replicates = replicates;
    a.r0 = replicate_offset;
    a.t = t;
    a.mode = functional;
    a.nsteps = nsteps;
    a.precision = precision;
    a.seed = seed;
    a.mean = mean;
    a.sem = sem;
    return from_cuda(launch_estimate_rqmc(p, a, st));
}

mcx_status mcx_estimate_noalloc(mcx_plan *p, const double *v, double t, int functional, int32_t nsteps,
                                uint64_t paths_per_entry, const int32_t *entries, int64_t n_entries, uint64_t seed,
                                uint64_t path_offset, int precision, double *mean, double *sem, void *stream) {
    NvtxRange nvtx("mcx_estimate_noalloc");
    mcx_status rc = check_common(p, t, functional, nsteps, precision);
    if (rc != MCX_OK) return rc;
    if (n_entries == 0) return MCX_OK;
    if (!v || n_entries < 0 || paths_per_entry < 1 || !mean) return MCX_E_INVALID;
    if (!entries && n_entries != p->n) return MCX_E_INVALID;
    if (paths_per_entry > (1ull << 53)) return MCX_E_INVALID;
    EstimateArgs a{};
    a.entries = entries;
    a.n_entries = n_entries;
    a.paths = paths_per_entry;
    a.t = t;
    a.mode = functional;
    a.nsteps = nsteps;
    a.precision = precision;
    a.seed = seed;
    a.path_offset = path_offset;
    a.mean = mean;
    a.sem = sem;
    bool too_large = false;
    cudaError_t e = launch_estimate_noalloc(p, v, a, static_cast<cudaStream_t>(stream), &too_large);
    if (too_large) return MCX_E_UNSUPPORTED;
    return from_cuda(e);
}

mcx_status mcx_estimate_forward(mcx_plan *p, const double *v, double t, int functional, int32_t nsteps,
                                uint64_t total_paths, uint64_t seed, uint64_t path_offset, int precision, double *x,
                                double *sem, void *stream) {
    NvtxRange nvtx("mcx_estimate_forward");
    mcx_status rc = check_common(p, t, functional, nsteps, precision);
    if (rc != MCX_OK) return rc;
    if (p->n == 0) return MCX_OK;
    if (!v || !x || total_paths < 1 || total_paths > (1ull << 53)) return MCX_E_INVALID;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (t == 0.0) {  // exp(0 A) v = v
        cudaError_t e = cudaMemcpyAsync(x, v, sizeof(double) * (size_t)p->n, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess && sem) e = cudaMemsetAsync(sem, 0, sizeof(double) * (size_t)p->n, st);
        return from_cuda(e);
    }
    return from_cuda(launch_estimate_forward(p, v, t, functional, nsteps, total_paths, seed, path_offset, precision,
                                             x, sem, st));
}

mcx_status mcx_total_communicability(mcx_plan *p, double t, int functional, int32_t nsteps, uint64_t total_paths,
                                     uint64_t seed, uint64_t path_offset, int precision, double *tc, double *sem,
                                     void *stream) {
    NvtxRange nvtx("mcx_total_communicability");
    mcx_status rc = check_common(p, t, functional, nsteps, precision);
    if (rc != MCX_OK) return rc;
    if (p->n == 0 || !tc || total_paths < 2 || total_paths > (1ull << 53)) return MCX_E_INVALID;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (t == 0.0) {  // 1^T 1 = n exactly
        const double nn = (double)p->n;
        cudaError_t e = cudaMemcpyAsync(tc, &nn, sizeof(double), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess && sem) e = cudaMemsetAsync(sem, 0, sizeof(double), st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // nn lives on this stack frame
        return from_cuda(e);
    }
    return from_cuda(launch_total_communicability(p, t, functional, nsteps, total_paths, seed, path_offset,
                                                  precision, tc, sem, st));
}

mcx_status mcx_trace_forward(mcx_plan *p, const double *v, double t, int functional, int32_t nsteps, uint64_t seed,
                             uint64_t first_path, uint32_t count, int precision, int32_t *start, int32_t *end,
                             uint32_t *njumps, uint64_t *hash, double *logw, void *stream) {
    NvtxRange nvtx("mcx_trace_forward");
    mcx_status rc = check_common(p, t, functional, nsteps, precision);
    if (rc != MCX_OK) return rc;
    if (!v || !start || !end || !njumps || !hash || !logw) return MCX_E_INVALID;
    return from_cuda(launch_trace_forward(p, v, t, functional, nsteps, seed, first_path, count, precision, start, end,
                                          njumps, hash, logw, static_cast<cudaStream_t>(stream)));
}

mcx_status mcx_trace_paths(mcx_plan *p, double t, int functional, int32_t nsteps, int32_t entry, uint64_t seed,
                           uint64_t first_path, uint32_t count, int precision, int32_t *end, uint32_t *njumps,
                           uint64_t *hash, double *logw, void *stream) {
    NvtxRange nvtx("mcx_trace_paths");
    mcx_status rc = check_common(p, t, functional, nsteps, precision);
    if (rc != MCX_OK) return rc;
    if (entry < 0 || entry >= p->n || !end || !njumps || !hash || !logw) return MCX_E_INVALID;
    return from_cuda(launch_trace(p, t, functional, nsteps, entry, seed, first_path, count, precision, end, njumps,
                                  hash, logw, static_cast<cudaStream_t>(stream)));
}

mcx_status mcx_power_iteration(int64_t n, const int64_t *row_ptr, const int32_t *col, const double *val,
                               int32_t max_iters, double tol, double *work, double *lambda_out, int32_t *iters_out,
                               void *stream) {
    NvtxRange nvtx("mcx_power_iteration");
    if (n <= 0 || !row_ptr || !col || !val || !work || max_iters < 1 || !(tol >= 0.0)) return MCX_E_INVALID;
    double lam = 0.0;
    int32_t it = 0;
    cudaError_t e = run_power_iteration(n, row_ptr, col, val, max_iters, tol, work, &lam, &it,
                                        static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return from_cuda(e);
    if (lambda_out) *lambda_out = lam;
    if (iters_out) *iters_out = it;
    return MCX_OK;
}

mcx_status mcx_expm_multiply(int64_t n, int64_t nnz, const int64_t *row_ptr, const int32_t *col, const double *val,
                             const double *v, double t, double beta_scale, int functional, int32_t nsteps,
                             uint64_t paths_per_entry, const int32_t *entries, int64_t n_entries, uint64_t seed,
                             uint64_t path_offset, int precision, uint32_t flags, double *mean, double *sem,
                             double *t_used, void *stream) {
    NvtxRange nvtx("mcx_expm_multiply");
    if (flags & ~MCX_PLAN_HOST_INPUT) return MCX_E_INVALID;
    if (n < 1 || nnz < 0 || !row_ptr || (nnz > 0 && (!col || !val)) || !v || !mean) return MCX_E_INVALID;
    if (!(t <= 0.0) && !(t > 0.0)) return MCX_E_INVALID;  // NaN
    if (t <= 0.0 && !(beta_scale > 0.0 && isfinite(beta_scale))) return MCX_E_INVALID;
    if (n_entries < 0 || (!entries && n_entries != n)) return MCX_E_INVALID;
    const bool host = (flags & MCX_PLAN_HOST_INPUT) != 0;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int64_t ne = entries ? n_entries : n;
    // device copies of the host arrays (pool); device arrays are used in place
    int64_t *d_rp = const_cast<int64_t *>(row_ptr);
    int32_t *d_col = const_cast<int32_t *>(col);
    double *d_val = const_cast<double *>(val), *d_v = const_cast<double *>(v), *d_mean = mean, *d_sem = sem;
    int32_t *d_ent = const_cast<int32_t *>(entries);
    double *work = nullptr;
    void *owned[8] = {};
    int n_owned = 0;
    mcx_plan *plan = nullptr;
    mcx_status rc = MCX_OK;
    cudaError_t e = cudaSuccess;
    auto take = [&](void **p, size_t bytes) {
        e = pool_alloc(p, bytes, st);
        if (e == cudaSuccess) owned[n_owned++] = *p;
        return e == cudaSuccess;
    };
    auto h2d = [&](void *dst, const void *src, size_t bytes) {
        e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st);
        return e == cudaSuccess;
    };
    do {
        if (host) {
            const size_t nz = (size_t)(nnz > 0 ? nnz : 1);
            if (!take(reinterpret_cast<void **>(&d_rp), 8 * (size_t)(n + 1)) ||
                !take(reinterpret_cast<void **>(&d_col), 4 * nz) || !take(reinterpret_cast<void **>(&d_val), 8 * nz) ||
                !take(reinterpret_cast<void **>(&d_v), 8 * (size_t)n) ||
                !take(reinterpret_cast<void **>(&d_mean), 8 * (size_t)(ne > 0 ? ne : 1)))
                break;
            if (sem && !take(reinterpret_cast<void **>(&d_sem), 8 * (size_t)(ne > 0 ? ne : 1))) break;
            if (entries && ne > 0 && !take(reinterpret_cast<void **>(&d_ent), 4 * (size_t)ne)) break;
            if (!h2d(d_rp, row_ptr, 8 * (size_t)(n + 1)) || (nnz > 0 && !h2d(d_col, col, 4 * (size_t)nnz)) ||
                (nnz > 0 && !h2d(d_val, val, 8 * (size_t)nnz)) || !h2d(d_v, v, 8 * (size_t)n) ||
                (entries && ne > 0 && !h2d(d_ent, entries, 4 * (size_t)ne)))
                break;
        }
        if ((rc = mcx_plan_create(n, nnz, d_rp, d_col, d_val, 0, stream, &plan)) != MCX_OK) break;
        if (t <= 0.0) {
            if (!take(reinterpret_cast<void **>(&work), 8 * (size_t)(3 * n + 4096))) break;
            double lam = 0.0;
            int32_t it = 0;
            if ((e = run_power_iteration(n, d_rp, d_col, d_val, 1000, 1e-10, work, &lam, &it, st)) != cudaSuccess)
                break;
            if (!(lam > 0.0) || !isfinite(lam)) {
                rc = MCX_E_INVALID;  // no positive dominant eigenvalue: beta = scale / lambda is undefined
                break;
            }
            t = beta_scale / lam;
        }
        if (t_used) *t_used = t;
        if ((rc = mcx_estimate(plan, d_v, t, functional, nsteps, paths_per_entry, entries ? d_ent : nullptr, ne, seed,
                               path_offset, precision, d_mean, d_sem, stream)) != MCX_OK)
            break;
        if (host && ne > 0) {
            if ((e = cudaMemcpyAsync(mean, d_mean, 8 * (size_t)ne, cudaMemcpyDeviceToHost, st)) != cudaSuccess) break;
            if (sem && (e = cudaMemcpyAsync(sem, d_sem, 8 * (size_t)ne, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
                break;
        }
        rc = mcx_sync(plan, stream, nullptr);  // synchronises the stream: the host results are complete
    } while (0);
    if (rc == MCX_OK && e != cudaSuccess) rc = from_cuda(e);
    for (int k = 0; k < n_owned; ++k) pool_free(owned[k], st);
    if (plan) {
        cudaStreamSynchronize(st);
        free_plan(plan);
    }
    return rc;
}

mcx_status mcx_plan_export(const mcx_plan *p, int32_t *deg, int64_t *row_start, uint8_t *weighted,
                           float *inv_rate32, float *delta32, double *inv_rate64, double *delta64, int32_t *edge_col,
                           int32_t *alias_col, uint32_t *thresh, void *stream) {
    if (!p) return MCX_E_INVALID;
    return from_cuda(launch_export(p, deg, row_start, weighted, inv_rate32, delta32, inv_rate64, delta64, edge_col,
                                   alias_col, thresh, static_cast<cudaStream_t>(stream)));
}

mcx_status mcx_sync(mcx_plan *p, void *stream, mcx_stats *stats) {
    NvtxRange nvtx("mcx_sync");
    if (!p) return MCX_E_INVALID;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    uint32_t hs[STATUS_SYNC_WORDS] = {0, 0, 0, 0, 0, 0, 0, 0};
    cudaError_t e = cudaMemcpyAsync(hs, p->status, 4 * STATUS_SYNC_WORDS, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return from_cuda(e);
    e = cudaMemsetAsync(p->status, 0, 4 * STATUS_SYNC_WORDS, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return from_cuda(e);
    if (stats) {
        stats->paths = ((uint64_t)hs[3] << 32) | hs[2];
        stats->jumps = ((uint64_t)hs[5] << 32) | hs[4];
        stats->status_bits = hs[0];
        stats->reserved = 0;
    }
    if (hs[0] & ST_BAD_ENTRY) return MCX_E_INVALID;
    if (hs[0] & ST_BAD_V) return MCX_E_NEG_V;
    return (hs[0] & ST_OVERFLOW) ? MCX_E_OVERFLOW : MCX_OK;
}

void mcx_plan_destroy(mcx_plan *p) {
    if (!p) return;
    cudaDeviceSynchronize();
    free_plan(p);
}

}  // extern "C"
