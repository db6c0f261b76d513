// Multilevel Monte Carlo over the time step (Giles 2008) for the STRANG and
// LIE functionals (Eqs. deff and eq_general1): the coupled level difference
// Y = v_{X_t} (W_N - W_{N/2}) evaluates the fine (N steps) and the coarse
// (N/2 steps) functional on the same continuous path.
//
// The draw schedule of a path does not depend on N (the path is simulated in
// continuous time and the potential is only sampled at the grid points), so
// the walker of walker.cuh runs the fine functional unchanged and this kernel
// keeps a second grid count beside it: a hold that starts with remaining time
// r0 in a state of potential delta and ends at r1 (or at the horizon) adds
// delta * (g_c(r0) - g_c(r1)) (or delta * g_c(r0)) with the coarse grid
// function g_c(rho) = min(N/2, floor(rho * N/(2t)) + 1), exactly what a walker
// with N/2 steps would add.  The difference is accumulated as
// e^{L_f} v (-expm1(L_c - L_f)), free of cancellation.
//
// Work decomposition and reduction follow the backward estimate: one warp per
// (entry, chunk) with lane refill and the staged entry row, log-shifted
// per-lane sums merged per warp, chunk partials merged per entry in chunk order.
#include <math.h>

#include <algorithm>

#include <type_traits>

#include "accum.cuh"
#include "launch.h"
#include "walker.cuh"

namespace mcx {
namespace {

struct DiffParams {
    int nc;                  // coarse steps N/2
    double dtc64, invdtc64;  // coarse step and its reciprocal
    float dtc32, invdtc32;
    Partial *part;           // [n_entries][chunks]
};

template <int MODE, bool WEIGHTED, bool F64>
__global__ void __launch_bounds__(WALK_THREADS, F64 ? WALK_MIN_BLOCKS_F64 : WALK_MIN_BLOCKS_F32)
    k_walk_diff(const __grid_constant__ WalkParams a, const DiffParams dp) {
    using Q = P<F64>;
    using T = typename Q::T;
    using Acc = typename std::conditional<F64, Acc64, Acc32>::type;
    __shared__ StageWarp s_stage[WARPS_PER_BLOCK];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const uint64_t wid = (uint64_t)blockIdx.x * WARPS_PER_BLOCK + warp;
    if (wid >= (uint64_t)a.n_entries * a.chunks_per_entry) return;  // warp-uniform; no block barrier
    const uint64_t e_idx = wid / a.chunks_per_entry;
    const uint64_t chunk = wid - e_idx * a.chunks_per_entry;
    const int32_t i = a.entries ? __ldg(a.entries + e_idx) : (int32_t)e_idx;
    if (i < 0 || (int64_t)i >= a.n) {  // invalid entry: flagged, NaN partial, nothing read
        if (lane == 0) {
            atomicOr(a.status, ST_BAD_ENTRY);
            dp.part[wid] = Partial{QNAN, 0.0, 0.0};
        }
        return;
    }
    const uint64_t p_begin = chunk * a.chunk_len;
    const uint64_t p_end = min(a.paths, p_begin + a.chunk_len);
    StageWarp &sw = s_stage[warp];
    const NodeRec start = load_node(a.node, i);
    const bool staged = !F64 && start.deg <= STAGE;
    if (lane == 0) sw.start = start;
    if (staged) stage_row<WEIGHTED>(sw, a, start, lane);
    __syncwarp();
    const StageWarp *swp = staged ? &sw : nullptr;
    const T delta_start = Q::pot(start, a.node64, i);
    const T t0 = F64 ? (T)a.t64 : (T)a.t32;
    const T invdtc = F64 ? (T)dp.invdtc64 : (T)dp.invdtc32;
    const T dtc = F64 ? (T)dp.dtc64 : (T)dp.dtc32;

    Walker<F64> w;
    w.rec = start; w.j = i; w.r = t0; w.acc = (T)0; w.delta = delta_start; w.k = 0;
    T accc = (T)0;  // coarse grid sum
    const uint64_t base = a.path_offset + p_begin;
    const uint32_t len = (uint32_t)(p_end - p_begin);
    uint32_t next = 32;
    uint32_t p = (uint32_t)lane;
    bool active = p < len;
    Acc acc;
    uint32_t jumps = 0;
    const unsigned lt_mask = (1u << lane) - 1u;
    while (__any_sync(0xffffffffu, active)) {
        bool fin = false;
        if (active) {
            const T r0 = w.r, d0 = w.delta;
            const uint64_t path = base + p;
            const uint4 rnd = philox_rk(make_uint4(w.k, (uint32_t)i, (uint32_t)path, (uint32_t)(path >> 32)), a);
            fin = advance_drawn<MODE, WEIGHTED, F64>(w, a, rnd, swp, i);
            const int gc = Q::grid(r0, invdtc, dp.nc) - (fin ? 0 : Q::grid(w.r, invdtc, dp.nc));
            accc = Q::fma(d0, Q::from_int(gc), accc);
            if (fin) {
                const T Lf = final_logw<MODE, F64>(w, delta_start, a);
                T Lc;
                if (MODE == MCX_LIE) {
                    Lc = Q::mul(accc, dtc);
                } else {
                    T s = Q::fma((T)0.5, delta_start, accc);
                    s = Q::fma((T)-0.5, w.delta, s);
                    Lc = Q::mul(s, dtc);
                }
                const T vend = F64 ? (T)__ldg(&a.node64[w.j].v) : (T)w.rec.v;
                T em1;
                if constexpr (F64) em1 = expm1(Lc - Lf);
                else em1 = expm1f(__fsub_rn(Lc, Lf));
                acc.add(Lf, -vend * em1);
                jumps += w.k;
            }
        }
        const unsigned fm = __ballot_sync(0xffffffffu, fin);
        if (fm) {
            if (fin) {
                p = next + (uint32_t)__popc(fm & lt_mask);
                active = p < len;
                w.rec = sw.start;
                w.j = i; w.r = t0; w.acc = (T)0; w.delta = delta_start; w.k = 0;
                accc = (T)0;
            }
            next += (uint32_t)__popc(fm);
        }
    }
    unsigned long long jl = jumps;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) jl += __shfl_xor_sync(0xffffffffu, jl, o);
    double S1, S2, Mw;
    acc.warp_merge(S1, S2, Mw);
    if (lane == 0) {
        unsigned long long *ctr = reinterpret_cast<unsigned long long *>(a.status + 2);
        atomicAdd(ctr, (unsigned long long)len);
        atomicAdd(ctr + 1, jl);
        dp.part[wid] = Partial{S1, S2, Mw};
    }
}

// One warp per entry: merge its chunk partials in chunk order, then mean and
// standard error.
__global__ void __launch_bounds__(WALK_THREADS) k_reduce_diff(const Partial *__restrict__ part, int64_t n_entries,
                                                             uint32_t cpe, double M, bool v_scaled, double *mean,
                                                             double *sem, uint32_t *status) {
    const int lane = threadIdx.x & 31;
    const int64_t e = ((int64_t)blockIdx.x * WALK_THREADS + threadIdx.x) >> 5;
    if (e >= n_entries) return;
    const Partial *pp = part + (uint64_t)e * cpe;
    bool bad = false;
    double m = -INFINITY;
    for (uint32_t c = lane; c < cpe; c += 32) {
        bad |= isnan(pp[c].s1);
        m = fmax(m, pp[c].m);
    }
    bad = __any_sync(0xffffffffu, bad);
    m = warp_max(m);
    double s1 = 0.0, s2 = 0.0;
    for (uint32_t c = lane; c < cpe; c += 32) {
        const Partial q = pp[c];
        const double sc = (q.m == -INFINITY) ? 0.0 : exp(q.m - m);
        s1 += sc * q.s1;
        s2 += sc * sc * q.s2;
    }
    s1 = warp_sum(s1);
    s2 = warp_sum(s2);
    if (lane == 0) {
        if (bad) {
            mean[e] = QNAN;
            if (sem) sem[e] = QNAN;
        } else {
            finish_entry(s1, s2, m, M, v_scaled ? v_scale(status) : 1.0, mean + e, sem ? sem + e : nullptr, status);
        }
    }
}

template <bool F64, bool WEIGHTED>
cudaError_t launch_diff_mode(int mode, unsigned grid, const WalkParams &p, const DiffParams &d, cudaStream_t st) {
    if (mode == MCX_STRANG) k_walk_diff<MCX_STRANG, WEIGHTED, F64><<<grid, WALK_THREADS, 0, st>>>(p, d);
    else k_walk_diff<MCX_LIE, WEIGHTED, F64><<<grid, WALK_THREADS, 0, st>>>(p, d);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_level_difference(mcx_plan *plan, const EstimateArgs &a, cudaStream_t st) {
    if (a.n_entries == 0) return cudaSuccess;
    WalkParams p = make_params(plan, a.t, a.nsteps, a.seed);
    p.entries = a.entries;
    p.n_entries = a.n_entries;
    p.paths = a.paths;
    p.path_offset = a.path_offset;
    DiffParams d{};
    d.nc = a.nsteps / 2;
    d.dtc64 = a.t / (double)d.nc;
    d.invdtc64 = (double)d.nc / a.t;
    d.dtc32 = (float)d.dtc64;
    d.invdtc32 = (float)d.invdtc64;
    // chunks as in the backward estimate: >= 1024 paths per warp, ~8 waves of warps
    const uint64_t target_warps = 152ull * 64ull * 8ull;
    uint64_t cpe = (target_warps + (uint64_t)a.n_entries - 1) / (uint64_t)a.n_entries;
    const uint64_t max_cpe = (a.paths + 1023) / 1024;
    if (cpe > max_cpe) cpe = max_cpe;
    if (cpe < 1) cpe = 1;
    if ((a.paths + cpe - 1) / cpe > (1ull << 30)) cpe = (a.paths + (1ull << 30) - 1) >> 30;
    uint64_t chunk = (a.paths + cpe - 1) / cpe;
    chunk = (chunk + 31) / 32 * 32;
    cpe = (a.paths + chunk - 1) / chunk;
    p.chunk_len = chunk;
    p.chunks_per_entry = (uint32_t)cpe;
    const uint64_t n_chunks = (uint64_t)a.n_entries * cpe;
    const uint64_t grid64 = (n_chunks + WARPS_PER_BLOCK - 1) / WARPS_PER_BLOCK;
    if (grid64 > 0x7FFFFFFFull) return cudaErrorInvalidValue;
    void *part = nullptr;
    cudaError_t e = pool_alloc(&part, sizeof(Partial) * (size_t)n_chunks, st);
    if (e != cudaSuccess) return e;
    d.part = static_cast<Partial *>(part);
    const bool weighted = plan->weighted_rows > 0;
    const unsigned grid = (unsigned)grid64;
    if (a.precision == MCX_FP64)
        e = weighted ? launch_diff_mode<true, true>(a.mode, grid, p, d, st)
                     : launch_diff_mode<true, false>(a.mode, grid, p, d, st);
    else
        e = weighted ? launch_diff_mode<false, true>(a.mode, grid, p, d, st)
                     : launch_diff_mode<false, false>(a.mode, grid, p, d, st);
    if (e == cudaSuccess) {
        const unsigned g2 = (unsigned)((a.n_entries + WARPS_PER_BLOCK - 1) / WARPS_PER_BLOCK);
        k_reduce_diff<<<g2, WALK_THREADS, 0, st>>>(d.part, a.n_entries, (uint32_t)cpe, (double)a.paths,
                                                   a.precision != MCX_FP64, a.mean, a.sem, plan->status);
        e = cudaGetLastError();
    }
    pool_free(part, st);
    return e;
}

}  // namespace mcx

namespace mcx {
namespace {

constexpr int MAX_LEVELS = 64;

struct LevelPtrs {
    const double *mean[MAX_LEVELS];
    const double *sem[MAX_LEVELS];
};

// Giles' telescoping sum per entry: the level means added in level order, the
// standard errors in quadrature (the levels use disjoint paths: independent).
__global__ void k_combine_levels(int32_t levels, int64_t n, const __grid_constant__ LevelPtrs p, double *mean,
                                 double *sem) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double m = 0.0, v = 0.0;
        for (int32_t l = 0; l < levels; ++l) {
            m += p.mean[l][i];
            if (sem) {
                const double s = p.sem[l][i];
                v = fma(s, s, v);
            }
        }
        mean[i] = m;
        if (sem) sem[i] = sqrt(v);
    }
}

}  // namespace
}  // namespace mcx

extern "C" mcx_status mcx_combine_levels(int32_t levels, int64_t n_entries, const double *const *means,
                                         const double *const *sems, double *mean, double *sem, void *stream) {
    using namespace mcx;
    if (levels < 1 || levels > MAX_LEVELS || n_entries < 0 || !means || !mean || (sem && !sems)) return MCX_E_INVALID;
    if (n_entries == 0) return MCX_OK;
    LevelPtrs p{};
    for (int32_t l = 0; l < levels; ++l) {
        if (!means[l] || (sem && !sems[l])) return MCX_E_INVALID;
        p.mean[l] = means[l];
        p.sem[l] = sem ? sems[l] : nullptr;
    }
    const unsigned grid = (unsigned)std::min<int64_t>((n_entries + 255) / 256, 152 * 8);
    k_combine_levels<<<grid, 256, 0, static_cast<cudaStream_t>(stream)>>>(levels, n_entries, p, mean, sem);
    return cudaGetLastError() == cudaSuccess ? MCX_OK : MCX_E_CUDA;
}
