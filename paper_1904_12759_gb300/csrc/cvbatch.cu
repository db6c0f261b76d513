// Batched backward full-vector estimates (Theorem 1, Algorithm 1) with the
// control variate of the variance-reduction remark of Sec. 5: many (A, v, t),
// several right-hand sides per A, one CUDA-graph launch per run.
//
// Layout.  The problems' matrices A_b go on the diagonal of one plan (blocks
// padded to multiples of 1024 states); each pair k = (problem b, right-hand
// side r), numbered problem by problem, owns a slot range of per-state arrays
// (its v, the FP32 copy of v scaled by a power of two, mean and standard
// error) and, with a control variate, its Taylor terms, features, prediction
// and coefficients.  Pair k simulates paths k * 2^40 + p of every entry with
// the entry's local index as the Philox stream word, so its paths are exactly
// those of the single-problem call (mcx_estimate / mcx_estimate_cv) with
// path_offset = k * 2^40: the walk runs on global state indices of the
// block-diagonal plan, whose rows are the problems' rows shifted by a
// constant, so every slot choice and every visited state is the same.
//
// Run (one graph launch).  Pre-pass over all pairs at once, on a CSR of the
// pairs' slots (each pair's copy of its problem's rows, columns shifted into
// its slots, each row with its pair's horizon) and a sliced ELL copy of its
// short rows: with a control variate three row passes (Av with the rates; A^2 v
// with the features; after the network's prediction on the tensor cores, A^3 v
// with A c3 and the coefficients), or the exponent and scaled FP32 copy of v
// for plain estimates.  Then one
// persistent walk over a work list in largest-estimated-cost-first order
// (cost ~ paths x (1 + t x mean jump rate)): pairs with at most 64 paths per
// entry take items of 32 entries with one lane per entry (all paths of the
// entry in path order, result written by the lane); the others take items
// (entry, chunk of paths) with one warp per item, lane refill, and the entry
// row staged in shared memory when the schedule says so; their chunk partials
// are merged per entry in chunk order by the finish kernel.  The seed is the
// only per-run parameter (the walk node's round keys are updated in the
// instantiated graph).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <string>
#include <type_traits>
#include <vector>

#include "accum.cuh"
#include "cvmath.cuh"
#include "expd.cuh"
#include "launch.h"
#include "rows.cuh"
#include "tune_cache.h"
#include "walker.cuh"

namespace mcx {
namespace {

constexpr int64_t CVB_BLOCK = 1024;        // plan blocks padded to multiples of this
constexpr int CVB_MIN_BLOCKS = 4;          // resident blocks per SM the plain walk is compiled for
constexpr int CVB_MIN_BLOCKS_CV = 3;       // and the control-variate walk (hold integrals need registers)
constexpr uint64_t CVB_ITEMS_PER_PAIR = 1ull << 20;  // chunk items per pair before chunks grow

struct CvbPair {
    int64_t off;         // first global state of the problem
    int64_t n;           // states (entries) of the problem
    int64_t slot;        // first per-state slot of this pair (every per-state array is slot-indexed)
    int64_t part0;       // first chunk partial (warp layout)
    uint64_t paths;      // paths per entry
    uint64_t path_base;  // pair index << 40
    uint64_t chunk;      // paths per chunk (warp layout)
    double t;
    float t32;
    uint32_t cpe;        // chunks per entry; 0: lane layout (paths <= LANE_MODE_MAX_PATHS)
    int32_t problem, rhs;
    double inv_m, inv_m1;  // 1/paths, 1/(paths - 1) (0 for one path)
    float inv_mf, inv_m1f;  // the same rounded to FP32
};

struct CvbItem {
    uint32_t pair;
    uint32_t e0;     // lane layout: first of 32 entries; warp layout: the entry
    uint32_t chunk;  // warp layout: chunk index
    uint32_t pad;
};

struct CvbArgs {
    const CvbPair *pairs;
    const CvbItem *items;
    uint32_t n_items;
    unsigned int *next_item;
    const double2 *ab;     // [slots] control-variate coefficients (a, b) of each pair's states
    const double *h;       // [slots] h(t) = the prediction of each pair's entries
    const float2 *abf;     // [slots] (a, b) 2^-k in FP32 (control variates with FP32 integrals)
    const double *v;       // [slots] float64 v of each pair (FP64 plain paths)
    const float *vf;       // [slots] v * 2^-vexp (FP32 plain paths)
    const uint32_t *vexp;  // [pairs] biased exponent: of v (plain FP32) or of the CV coefficients (FP32 integrals)
    Partial *part;
    double *mean, *sem;    // [slots]
};

// Per-pair biased exponent of the largest finite |x| over the pair's slots, `per`
// doubles per slot (1 for v, 2 for the coefficient pairs); the words are cleared
// first.  A warp takes 32 consecutive slots, mostly of one pair, and keeps a
// running maximum while its pair stays the same: one atomic per warp and pair
// then, one per lane where a pair boundary falls inside the 32 slots.
__global__ void k_pair_exponent(int64_t slots, int per, const double *__restrict__ x,
                                const int32_t *__restrict__ slot_pair, uint32_t *vexp) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    uint32_t acc = 0;  // the warp's running maximum for pair acc_k (warp-uniform)
    int32_t acc_k = -1;
    for (int64_t w0 = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32; w0 < slots; w0 += warps * 32) {
        const int64_t s = w0 + lane;
        uint32_t e = 0;
        int32_t k = -1;
        if (s < slots) {
            k = slot_pair[s];
            for (int q = 0; q < per; ++q) {  // ilogb of finite nonzero values, from the bits
                const unsigned long long y =
                    (unsigned long long)__double_as_longlong(x[s * per + q]) & 0x7fffffffffffffffull;
                if (y != 0ull && y < 0x7ff0000000000000ull) {
                    const int E = (int)(y >> 52);
                    const int lg = E ? E - 1023 : (63 - __clzll((long long)y)) - 1074;
                    e = max(e, (uint32_t)(lg + (int)VEXP_BIAS));
                }
            }
        }
        const int32_t k0 = __shfl_sync(0xffffffffu, k, 0);
        if (__all_sync(0xffffffffu, k == k0 || k < 0)) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, o));
            if (k0 == acc_k) {
                acc = max(acc, e);
            } else {
                if (lane == 0 && acc) atomicMax(vexp + acc_k, acc);
                acc_k = k0;
                acc = e;
            }
        } else if (k >= 0 && e) {
            atomicMax(vexp + k, e);
        }
    }
    if (lane == 0 && acc) atomicMax(vexp + acc_k, acc);
}

// FP32 copies scaled by the pair's power of two: v (plain) and the coefficient pairs.
__global__ void k_pair_pack(int64_t slots, const double *__restrict__ v, const int32_t *__restrict__ slot_pair,
                            const uint32_t *__restrict__ vexp, float *__restrict__ vf) {
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < slots; s += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t eb = vexp[slot_pair[s]];
        vf[s] = __double2float_rn(ldexp(v[s], eb ? -((int)eb - (int)VEXP_BIAS) : 0));
    }
}

__global__ void k_pair_coef_f32(int64_t slots, const double2 *__restrict__ ab, const int32_t *__restrict__ slot_pair,
                                const uint32_t *__restrict__ vexp, float2 *__restrict__ out) {
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < slots; s += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t eb = vexp[slot_pair[s]];
        const int k = eb ? (int)eb - (int)VEXP_BIAS : 0;
        const double2 c = ab[s];
        if (k >= -1022 && k <= 1022) {  // 2^-k a normal number: one exact product each
            const double p2 = __longlong_as_double((long long)(1023 - k) << 52);
            out[s] = make_float2(__double2float_rn(__dmul_rn(c.x, p2)), __double2float_rn(__dmul_rn(c.y, p2)));
        } else {
            out[s] = make_float2(__double2float_rn(ldexp(c.x, -k)), __double2float_rn(ldexp(c.y, -k)));
        }
    }
}

// The lane sums of a control-variate walker: FP64 plain sums of the per-path
// residual integrals, or FP32 shifted compensated sums of e^{Ls} ys.
template <bool F64I>
struct CvLane {
    double s1 = 0.0, s2 = 0.0;
    float m = -INFINITY, f1 = 0.f, c1 = 0.f, f2 = 0.f;
    using R = typename std::conditional<F64I, double, float>::type;
    __device__ __forceinline__ void end_path(R ys, float Ls) {
        if (F64I) {
            s1 += (double)ys;
            s2 += (double)ys * (double)ys;
        } else {
            if (!(Ls <= m + 8.0f)) {
                const float sc = (m == -INFINITY) ? 0.0f : expf(m - Ls);
                f1 *= sc; c1 *= sc; f2 *= sc * sc;
                m = Ls;
            }
            const float wv = __fmul_rn(expf(__fsub_rn(Ls, m)), (float)ys);
            const float yk = __fsub_rn(wv, c1);
            const float tk = __fadd_rn(f1, yk);
            c1 = __fsub_rn(__fsub_rn(tk, f1), yk);
            f1 = tk;
            f2 = __fmaf_rn(wv, wv, f2);
        }
    }
    __device__ __forceinline__ void result(double &S1, double &S2, double &M) const {
        if (F64I) {
            S1 = s1; S2 = s2; M = 0.0;
        } else {
            S1 = (double)f1 - (double)c1; S2 = (double)f2; M = (double)m;
        }
    }
    __device__ __forceinline__ void warp_merge(double &S1, double &S2, double &M) const {
        if (F64I) {
            S1 = warp_sum(s1); S2 = warp_sum(s2); M = 0.0;
        } else {
            float mw = m;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) mw = fmaxf(mw, __shfl_xor_sync(0xffffffffu, mw, o));
            const double sc = (m == -INFINITY) ? 0.0 : exp((double)m - (double)mw);
            S1 = warp_sum(sc * ((double)f1 - (double)c1));
            S2 = warp_sum(sc * sc * (double)f2);
            M = (double)mw;
        }
    }
};

// One event of a control-variate path: advance, then add the hold's residual
// integral e^{L0} int R to the path's running sum (ys with shift Ls in FP32).
// FP64 integrals read the coefficient pairs from ab, FP32 ones the scaled FP32
// copy abf (see k_coef_f32); both indexed by the state's offset in its problem.
template <bool F64I, bool WEIGHTED>
__device__ __forceinline__ bool cv_event(Walker<false> &w, const WalkParams &a, uint32_t stream, uint64_t path,
                                         const StageWarp *sw, int32_t i0, const double2 *__restrict__ ab,
                                         const float2 *__restrict__ abf, int64_t off,
                                         typename CvLane<F64I>::R &ys, float &Ls) {
    using R = typename CvLane<F64I>::R;
    const int32_t j = w.j;
    const float r0 = w.r, L0 = w.acc, dl = w.delta;
    float D;
    const bool fin = advance<MCX_EXACT, WEIGHTED, false>(w, a, stream, path, sw, i0, &D);
    R ca, cb;
    if constexpr (F64I) {
        const double2 c = __ldg(ab + (j - off));
        ca = c.x;
        cb = c.y;
    } else {
        const float2 c = __ldg(abf + (j - off));
        ca = c.x;
        cb = c.y;
    }
    const R J = hold_integral<R>(ca, cb, (R)dl, (R)r0, (R)D);
    if (F64I) {
        ys += (R)exp((double)L0) * J;
    } else {
        if (L0 > Ls + 40.0f) {  // keep e^{L - Ls} in range
            ys *= (R)expf(Ls - L0);
            Ls = L0;
        }
        ys += (R)expf(L0 - Ls) * J;
    }
    return fin;
}

// x finite, by its exponent bits (integer pipe)
__device__ __forceinline__ bool finite_bits(double x) {
    return ((unsigned long long)__double_as_longlong(x) & 0x7ff0000000000000ull) != 0x7ff0000000000000ull;
}

// The persistent walk.  CV: control variate (FP32 paths; F64: residual
// integrals in FP64); plain: F64 selects the FP64 path version.
template <bool CV, bool F64, bool WEIGHTED, bool STAGED>
__global__ void __launch_bounds__(WALK_THREADS, CV ? CVB_MIN_BLOCKS_CV : CVB_MIN_BLOCKS)
    k_cvb_walk(const __grid_constant__ WalkParams a, const __grid_constant__ CvbArgs b) {
    constexpr bool P64 = F64 && !CV;  // FP64 paths (plain only)
    using Q = P<P64>;
    using T = typename Q::T;
    using Acc = typename std::conditional<P64, Acc64, Acc32>::type;
    using R = typename CvLane<F64>::R;
    __shared__ StageWarp s_stage[STAGED ? WARPS_PER_BLOCK : 1];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const unsigned lt_mask = (1u << lane) - 1u;
    unsigned long long paths_done = 0, jumps_done = 0;
    for (;;) {
        unsigned int item = 0;
        if (lane == 0) item = atomicAdd(b.next_item, 1u);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= b.n_items) break;
        const CvbItem it = b.items[item];
        const CvbPair pr = b.pairs[it.pair];
        const double2 *ab = CV ? b.ab + pr.slot : nullptr;
        const float2 *abf = (CV && !F64) ? b.abf + pr.slot : nullptr;
        // FP32 residual integrals: coefficients scaled by 2^-k (k from the pre-pass), results by 2^k
        const double up = (CV && !F64) ? exp_scale(b.vexp[it.pair]) : 1.0;
        const T t0 = P64 ? (T)pr.t : (T)pr.t32;
        if (pr.cpe == 0) {
            // ---- lane layout: lane = entry, all paths in path order ----
            const int64_t e = (int64_t)it.e0 + lane;
            if (e < pr.n) {
                const int32_t i0 = (int32_t)(pr.off + e);
                const NodeRec start = load_node(a.node, i0);
                const T delta_start = Q::pot(start, a.node64, i0);
                Acc acc;
                CvLane<F64> cl;
                for (uint64_t p = 0; p < pr.paths; ++p) {
                    const uint64_t path = pr.path_base + p;
                    if constexpr (CV) {
                        Walker<false> w;
                        w.rec = start; w.j = i0; w.r = pr.t32; w.acc = 0.0f; w.delta = start.delta; w.k = 0;
                        R ys = (R)0;
                        float Ls = 0.0f;
                        while (!cv_event<F64, WEIGHTED>(w, a, (uint32_t)e, path, nullptr, i0, ab, abf, pr.off, ys,
                                                        Ls)) {
                        }
                        cl.end_path(ys, Ls);
                        jumps_done += w.k;
                    } else {
                        Walker<P64> w;
                        w.rec = start; w.j = i0; w.r = t0; w.acc = (T)0; w.delta = delta_start; w.k = 0;
                        while (!advance<MCX_EXACT, WEIGHTED, P64>(w, a, (uint32_t)e, path, nullptr, i0)) {
                        }
                        const int64_t s = pr.slot + (w.j - pr.off);
                        if (P64) acc.add(w.acc, (T)__ldg(b.v + s));
                        else acc.add(w.acc, (T)__ldg(b.vf + s));
                        jumps_done += w.k;
                    }
                }
                paths_done += pr.paths;
                const double M = (double)pr.paths;
                double S1, S2, Mw;
                const int ku = b.vexp[it.pair] ? (int)b.vexp[it.pair] - (int)VEXP_BIAS : 0;
                if (CV && !F64 && cl.m >= -40.0f && cl.m <= 40.0f && ku >= -60 && ku <= 60) {
                    // FP32 integrals, one entry per lane, scale e^m 2^k inside the FP32
                    // range: the residual mean and standard error in FP32 (the sums are
                    // FP32 already; GB300 runs FP64 slowly), added to h in FP64
                    const float sc = __fmul_rn(expf(cl.m), __uint_as_float((uint32_t)(ku + 127) << 23));
                    const float s1 = __fsub_rn(cl.f1, cl.c1);
                    const float muf = __fmul_rn(s1, pr.inv_mf);
                    float varf = __fmul_rn(__fsub_rn(cl.f2, __fmul_rn(s1, muf)), pr.inv_m1f);
                    if (!(varf > 0.0f)) varf = 0.0f;
                    const double mv = b.h[pr.slot + e] + (double)__fmul_rn(sc, muf);
                    const double se = (double)__fmul_rn(sc, __fsqrt_rn(__fmul_rn(varf, pr.inv_mf)));
                    b.mean[pr.slot + e] = mv;
                    b.sem[pr.slot + e] = se;
                    if (!finite_bits(mv) || !finite_bits(se)) atomicOr(a.status, ST_OVERFLOW);
                } else if constexpr (CV && !F64) {
                    // FP32 integrals with a scale outside that range: the few FP64 operations
                    // of the finish -- e^Mw of the FP32 maximum by the table-driven
                    // exponential, the divisions by M as products with the pair's
                    // reciprocals, the standard error's root in FP32 where its argument is
                    // well inside the FP32 range (relative error 2^-23)
                    cl.result(S1, S2, Mw);
                    const float mf = (float)Mw;
                    const double scale = (mf == -INFINITY ? 0.0 : exp_of_f32(mf)) * up;
                    const double mu = S1 * pr.inv_m;
                    double var = (S2 - S1 * mu) * pr.inv_m1;
                    if (!(var > 0.0)) var = 0.0;
                    const double q = var * pr.inv_m;
                    const double mv = b.h[pr.slot + e] + scale * mu;
                    const double se = scale * ((q > 1e-30 && q < 1e30) ? (double)__fsqrt_rn((float)q)
                                                                       : (q > 0.0 ? sqrt(q) : 0.0));
                    b.mean[pr.slot + e] = mv;
                    b.sem[pr.slot + e] = se;
                    if (!finite_bits(mv) || !finite_bits(se)) atomicOr(a.status, ST_OVERFLOW);
                } else if constexpr (CV) {
                    cl.result(S1, S2, Mw);
                    const double scale = ((Mw == -INFINITY) ? 0.0 : exp(Mw)) * up;
                    const double mu = S1 / M;
                    double var = M > 1.0 ? (S2 - S1 * mu) / (M - 1.0) : 0.0;
                    if (var < 0.0) var = 0.0;
                    const double mv = b.h[pr.slot + e] + scale * mu;
                    const double se = scale * sqrt(var / M);
                    b.mean[pr.slot + e] = mv;
                    b.sem[pr.slot + e] = se;
                    if (!isfinite(mv) || !isfinite(se)) atomicOr(a.status, ST_OVERFLOW);
                } else {
                    acc.lane_result(S1, S2, Mw);
                    const double vs = P64 ? 1.0 : ldexp(1.0, b.vexp[it.pair] ? (int)b.vexp[it.pair] - (int)VEXP_BIAS : 0);
                    finish_entry(S1, S2, Mw, M, vs, b.mean + pr.slot + e, b.sem + pr.slot + e, a.status);
                }
            }
            continue;
        }
        // ---- warp layout: one entry, one chunk of its paths, lane refill ----
        const int64_t e = it.e0;
        const int32_t i0 = (int32_t)(pr.off + e);
        const uint64_t p_begin = (uint64_t)it.chunk * pr.chunk;
        const uint32_t len = (uint32_t)(min(pr.paths, p_begin + pr.chunk) - p_begin);
        const uint64_t base = pr.path_base + p_begin;
        const NodeRec start = load_node(a.node, i0);
        StageWarp &sw = s_stage[STAGED ? warp : 0];
        const bool staged = STAGED && !P64 && start.deg <= STAGE;
        if (STAGED) {
            __syncwarp();  // the previous item's reads of the staged row are done
            if (lane == 0) sw.start = start;
            if (staged) stage_row<WEIGHTED>(sw, a, start, lane);
            __syncwarp();
        }
        const StageWarp *swp = staged ? &sw : nullptr;
        const T delta_start = Q::pot(start, a.node64, i0);
        uint32_t next = 32, p = (uint32_t)lane;
        bool active = p < len;
        uint32_t jumps = 0;
        double S1, S2, Mw;
        if constexpr (CV) {
            Walker<false> w;
            w.rec = start; w.j = i0; w.r = pr.t32; w.acc = 0.0f; w.delta = start.delta; w.k = 0;
            R ys = (R)0;
            float Ls = 0.0f;
            CvLane<F64> cl;
            while (__any_sync(0xffffffffu, active)) {
                bool fin = false;
                if (active && cv_event<F64, WEIGHTED>(w, a, (uint32_t)e, base + p, swp, i0, ab, abf, pr.off, ys, Ls)) {
                    fin = true;
                    cl.end_path(ys, Ls);
                    jumps += w.k;
                }
                const unsigned fm = __ballot_sync(0xffffffffu, fin);
                if (fm) {
                    if (fin) {
                        p = next + (uint32_t)__popc(fm & lt_mask);
                        active = p < len;
                        w.rec = start; w.j = i0; w.r = pr.t32; w.acc = 0.0f; w.delta = start.delta; w.k = 0;
                        ys = (R)0;
                        Ls = 0.0f;
                    }
                    next += (uint32_t)__popc(fm);
                }
            }
            cl.warp_merge(S1, S2, Mw);
        } else {
            Walker<P64> w;
            w.rec = start; w.j = i0; w.r = t0; w.acc = (T)0; w.delta = delta_start; w.k = 0;
            Acc acc;
            while (__any_sync(0xffffffffu, active)) {
                bool fin = false;
                if (active && advance<MCX_EXACT, WEIGHTED, P64>(w, a, (uint32_t)e, base + p, swp, i0)) {
                    fin = true;
                    const int64_t s = pr.slot + (w.j - pr.off);
                    if (P64) acc.add(w.acc, (T)__ldg(b.v + s));
                    else acc.add(w.acc, (T)__ldg(b.vf + s));
                    jumps += w.k;
                }
                const unsigned fm = __ballot_sync(0xffffffffu, fin);
                if (fm) {
                    if (fin) {
                        p = next + (uint32_t)__popc(fm & lt_mask);
                        active = p < len;
                        w.rec = start; w.j = i0; w.r = t0; w.acc = (T)0; w.delta = delta_start; w.k = 0;
                    }
                    next += (uint32_t)__popc(fm);
                }
            }
            acc.warp_merge(S1, S2, Mw);
        }
        unsigned long long jl = jumps;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) jl += __shfl_xor_sync(0xffffffffu, jl, o);
        if (lane == 0) {
            b.part[pr.part0 + e * pr.cpe + it.chunk] = Partial{S1, S2, Mw};
            paths_done += len;
            jumps_done += jl;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        jumps_done += __shfl_xor_sync(0xffffffffu, jumps_done, o);
        paths_done += __shfl_xor_sync(0xffffffffu, paths_done, o);
    }
    if (lane == 0 && paths_done) {
        unsigned long long *ctr = reinterpret_cast<unsigned long long *>(a.status + 2);
        atomicAdd(ctr, paths_done);
        atomicAdd(ctr + 1, jumps_done);
    }
}

// Warp-layout pairs: per entry, merge the chunk partials in chunk order; mean
// = h_i + e^m S1/M (control variate) or e^m S1/M times the v scale (plain).
__global__ void k_cvb_finish(const CvbPair *__restrict__ pairs, const int32_t *__restrict__ warp_pairs, bool cv,
                             bool scaled, CvbArgs b, uint32_t *status) {
    const int32_t k = warp_pairs[blockIdx.y];
    const CvbPair pr = pairs[k];
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= pr.n) return;
    const Partial *pp = b.part + pr.part0 + e * pr.cpe;
    double mx = -INFINITY;
    for (uint32_t c = 0; c < pr.cpe; ++c) mx = fmax(mx, pp[c].m);
    double s1 = 0.0, s2 = 0.0;
    for (uint32_t c = 0; c < pr.cpe; ++c) {
        const Partial q = pp[c];
        const double sc = (q.m == -INFINITY) ? 0.0 : exp(q.m - mx);
        s1 += sc * q.s1;
        s2 += sc * sc * q.s2;
    }
    const double M = (double)pr.paths;
    if (cv) {
        // FP32 residual integrals carry the coefficients' power-of-two scale (word 0 otherwise)
        const double scale = (mx == -INFINITY ? 0.0 : exp(mx)) * exp_scale(b.vexp[k]);
        const double mu = s1 / M;
        double var = M > 1.0 ? (s2 - s1 * mu) / (M - 1.0) : 0.0;
        if (var < 0.0) var = 0.0;
        const double mv = b.h[pr.slot + e] + scale * mu;
        const double se = scale * sqrt(var / M);
        b.mean[pr.slot + e] = mv;
        b.sem[pr.slot + e] = se;
        if (!isfinite(mv) || !isfinite(se)) atomicOr(status, ST_OVERFLOW);
    } else {
        const uint32_t eb = b.vexp[k];
        const double vs = scaled ? ldexp(1.0, eb ? (int)eb - (int)VEXP_BIAS : 0) : 1.0;
        finish_entry(s1, s2, mx, M, vs, b.mean + pr.slot + e, b.sem + pr.slot + e, status);
    }
}

template <bool CV, bool F64, bool WEIGHTED, bool STAGED>
void *walk_fn() {
    return (void *)k_cvb_walk<CV, F64, WEIGHTED, STAGED>;
}

void *pick_walk(bool cv, bool f64, bool weighted, bool staged) {
    void *(*table[16])() = {
        walk_fn<false, false, false, false>, walk_fn<false, false, false, true>, walk_fn<false, false, true, false>,
        walk_fn<false, false, true, true>,   walk_fn<false, true, false, false>,  walk_fn<false, true, false, true>,
        walk_fn<false, true, true, false>,   walk_fn<false, true, true, true>,    walk_fn<true, false, false, false>,
        walk_fn<true, false, false, true>,   walk_fn<true, false, true, false>,   walk_fn<true, false, true, true>,
        walk_fn<true, true, false, false>,   walk_fn<true, true, false, true>,    walk_fn<true, true, true, false>,
        walk_fn<true, true, true, true>};
    return table[(cv ? 8 : 0) + (f64 ? 4 : 0) + (weighted ? 2 : 0) + (staged ? 1 : 0)]();
}

}  // namespace
}  // namespace mcx

using namespace mcx;

struct mcx_cvbatch {
    int32_t problems = 0;
    int32_t n_pair = 0;
    int control = MCX_CV_NONE;
    int precision = MCX_FP32;
    const mcx_mlp *net = nullptr;
    int64_t N = 0;        // padded states
    int64_t slots = 0;    // sum over pairs of n_b
    mcx_plan *plan = nullptr;
    std::vector<CvbPair> pair_host;
    std::vector<double> cost_per_path;  // per pair
    std::vector<uint64_t> paths;        // per problem
    // the pre-pass's CSR over slots (control variates): each pair's copy of its
    // problem's rows, columns shifted to the pair's slots, so that one pass
    // prepares every pair
    int64_t *srp = nullptr;     // [slots + 1]
    int32_t *scol = nullptr;
    double *sval = nullptr;
    int32_t *sorder = nullptr;   // [slots] its row schedule (built once, on the host)
    uint32_t *scnt = nullptr;    // [CV_ROW_CNT] the schedule's counts
    int32_t *ell_col = nullptr;  // sliced ELL copy of its short rows (see CvSell)
    double *ell_val = nullptr;
    int64_t *ell_chunk = nullptr;
    uint8_t *ell_len = nullptr;
    double *t_row = nullptr;    // [2 slots] horizon t of each slot's pair, then 1/(t*t*t)
    int32_t *slot_pair = nullptr;  // [slots] pair of each slot
    // per-slot arrays
    double *v = nullptr;      // [slots]
    float *vf = nullptr;      // [slots]
    uint32_t *vexp = nullptr;  // [pairs]
    double *taylor = nullptr;  // [4 slots]
    float *feat = nullptr;     // [5 slots]
    float *y = nullptr;        // [slots]
    double2 *ab = nullptr;     // [slots] coefficient pairs
    double *h = nullptr;       // [slots] predictions h(t)
    float2 *abf = nullptr;     // [slots] scaled FP32 coefficient pairs (FP32 integrals)
    double *work = nullptr;    // [2 slots] 16-byte records of the row passes
    double *mean = nullptr, *sem = nullptr;  // [slots]
    CvbPair *pairs = nullptr;
    int32_t *warp_pairs = nullptr;
    int32_t n_warp_pairs = 0;
    int64_t warp_pairs_max_n = 0;
    Partial *part = nullptr;
    int64_t part_cap = 0;
    CvbItem *items = nullptr;
    uint64_t items_cap = 0;
    uint32_t n_items = 0;
    unsigned int *next_item = nullptr;
    uint32_t chunk = 2048;
    int blocks_per_sm = CVB_MIN_BLOCKS;
    bool staged = true;
    int sms = 0;
    double tuned_ms = 0.0;
    WalkParams wp{};
    CvbArgs ba{};
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphNode_t walk_node = nullptr;
};

namespace {

mcx_status cvb_status(cudaError_t e) {
    if (e == cudaSuccess) return MCX_OK;
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return MCX_E_OOM;
    }
    return MCX_E_CUDA;
}

void free_cvbatch(mcx_cvbatch *b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    void *bufs[] = {b->srp, b->scol, b->sval, b->sorder, b->scnt, b->ell_col, b->ell_val, b->ell_chunk, b->ell_len,
                    b->t_row, b->slot_pair, b->v, b->vf, b->vexp, b->taylor, b->feat, b->y,
                    b->ab, b->h, b->abf, b->work,
                    b->mean, b->sem, b->pairs, b->warp_pairs, b->part, b->items, b->next_item};
    for (void *p : bufs) dev_free(p);
    if (b->plan) mcx_plan_destroy(b->plan);
    delete b;
}

bool cv_mode(const mcx_cvbatch *b) { return b->control != MCX_CV_NONE; }

// Per-pair layout for the current paths and chunk length: lane or warp layout,
// chunks per entry, partial offsets.  Host only.
void layout_pairs(mcx_cvbatch *b) {
    int64_t part = 0;
    for (auto &pr : b->pair_host) {
        pr.paths = b->paths[pr.problem];
        pr.inv_m = 1.0 / (double)pr.paths;
        pr.inv_m1 = pr.paths > 1 ? 1.0 / (double)(pr.paths - 1) : 0.0;
        pr.inv_mf = (float)pr.inv_m;
        pr.inv_m1f = (float)pr.inv_m1;
        if (pr.paths <= LANE_MODE_MAX_PATHS) {
            pr.cpe = 0;
            pr.chunk = pr.paths;
            pr.part0 = 0;
            continue;
        }
        uint64_t cpe = (pr.paths + b->chunk - 1) / b->chunk;
        const uint64_t cap = std::max<uint64_t>(1, CVB_ITEMS_PER_PAIR / (uint64_t)pr.n);
        if (cpe > cap) cpe = cap;
        const uint64_t min_cpe = (pr.paths + (1ull << 30) - 1) >> 30;  // chunks below 2^30 paths
        if (cpe < min_cpe) cpe = min_cpe;
        uint64_t chunk = (pr.paths + cpe - 1) / cpe;
        chunk = (chunk + 31) / 32 * 32;
        cpe = (pr.paths + chunk - 1) / chunk;
        pr.cpe = (uint32_t)cpe;
        pr.chunk = chunk;
        pr.part0 = part;
        part += pr.n * (int64_t)cpe;
    }
}

int64_t partials_needed(const mcx_cvbatch *b) {
    int64_t part = 0;
    for (const auto &pr : b->pair_host)
        if (pr.cpe) part += pr.n * (int64_t)pr.cpe;
    return part;
}

// Items of the current layout in largest-estimated-cost-first order; with
// stride > 1 only every stride-th (the autotuner's sample).
std::vector<CvbItem> make_items(const mcx_cvbatch *b, uint32_t stride) {
    std::vector<int32_t> order(b->n_pair);
    for (int32_t k = 0; k < b->n_pair; ++k) order[k] = k;
    auto item_cost = [b](int32_t k) {
        const CvbPair &p = b->pair_host[k];
        const double paths = p.cpe ? (double)p.chunk : 32.0 * (double)p.paths;
        return paths * b->cost_per_path[k];
    };
    std::stable_sort(order.begin(), order.end(), [&](int32_t x, int32_t y) { return item_cost(x) > item_cost(y); });
    std::vector<CvbItem> items;
    uint64_t idx = 0;
    for (int32_t k : order) {
        const CvbPair &p = b->pair_host[k];
        if (p.cpe == 0) {
            for (int64_t e = 0; e < p.n; e += 32, ++idx)
                if (idx % stride == 0) items.push_back(CvbItem{(uint32_t)k, (uint32_t)e, 0u, 0u});
        } else {
            for (int64_t e = 0; e < p.n; ++e)
                for (uint32_t c = 0; c < p.cpe; ++c, ++idx)
                    if (idx % stride == 0) items.push_back(CvbItem{(uint32_t)k, (uint32_t)e, c, 0u});
        }
    }
    return items;
}

cudaError_t upload_items(mcx_cvbatch *b, const std::vector<CvbItem> &items, cudaStream_t st) {
    cudaError_t e = cudaSuccess;
    if (items.size() + 1 > b->items_cap) {
        dev_free(b->items);
        b->items = nullptr;
        b->items_cap = 0;
        if ((e = dev_malloc(reinterpret_cast<void **>(&b->items), sizeof(CvbItem) * (items.size() + 1))) !=
            cudaSuccess)
            return e;
        b->items_cap = items.size() + 1;
    }
    if (!items.empty())
        e = cudaMemcpyAsync(b->items, items.data(), sizeof(CvbItem) * items.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    b->n_items = (uint32_t)items.size();
    b->ba.items = b->items;
    b->ba.n_items = b->n_items;
    return e;
}

// Apply a new layout on the device: pairs, partials, warp-pair list, full item list.
cudaError_t apply_layout(mcx_cvbatch *b, cudaStream_t st) {
    layout_pairs(b);
    cudaError_t e;
    const int64_t need = partials_needed(b);
    if (need + 1 > b->part_cap) {
        dev_free(b->part);
        b->part = nullptr;
        b->part_cap = 0;
        if ((e = dev_malloc(reinterpret_cast<void **>(&b->part), sizeof(Partial) * (size_t)(need + 1))) != cudaSuccess)
            return e;
        b->part_cap = need + 1;
    }
    std::vector<int32_t> wp;
    int64_t mx = 0;
    for (int32_t k = 0; k < b->n_pair; ++k)
        if (b->pair_host[k].cpe) {
            wp.push_back(k);
            mx = std::max(mx, b->pair_host[k].n);
        }
    b->n_warp_pairs = (int32_t)wp.size();
    b->warp_pairs_max_n = mx;
    if ((e = cudaMemcpyAsync(b->pairs, b->pair_host.data(), sizeof(CvbPair) * b->n_pair, cudaMemcpyHostToDevice,
                             st)) != cudaSuccess)
        return e;
    if (!wp.empty() &&
        (e = cudaMemcpyAsync(b->warp_pairs, wp.data(), sizeof(int32_t) * wp.size(), cudaMemcpyHostToDevice, st)) !=
            cudaSuccess)
        return e;
    b->ba.part = b->part;
    const uint64_t total = [&]() {
        uint64_t s = 0;
        for (const auto &p : b->pair_host) s += p.cpe ? (uint64_t)p.n * p.cpe : (uint64_t)((p.n + 31) / 32);
        return s;
    }();
    if (total >= (1ull << 31)) return cudaErrorInvalidValue;
    return upload_items(b, make_items(b, 1), st);
}

// The row schedule of the pre-pass's CSR and the sliced ELL copy of its short
// rows (see CvSell), built on the host: huge rows, long rows, then the short
// rows in natural order, so that a chunk's 32 rows are neighbours and their
// per-row reads and writes fall in few sectors (sorting rows by length within
// windows of 64..256 rows, to keep every lane busy, measured slower on GB300).
// Padding slots of a chunk are zero and never read.
struct HostEll {
    std::vector<int32_t> order, col;
    std::vector<double> val;
    std::vector<int64_t> chunk;
    std::vector<uint8_t> len;
    uint32_t cnt[CV_ROW_CNT] = {};
};

void build_ell(int64_t n, const std::vector<int64_t> &rp, const std::vector<int32_t> &col,
               const std::vector<double> &val, HostEll &E) {
    std::vector<int32_t> huge, lng, shrt;
    for (int64_t i = 0; i < n; ++i) {
        const int64_t len = rp[i + 1] - rp[i];
        if (len > HUGE_ROW) huge.push_back((int32_t)i);
        else if (len > LONG_ROW) lng.push_back((int32_t)i);
        else shrt.push_back((int32_t)i);
    }
    E.cnt[0] = (uint32_t)huge.size();
    E.cnt[1] = (uint32_t)lng.size();
    E.cnt[2] = (uint32_t)shrt.size();
    E.order.reserve((size_t)std::max<int64_t>(n, 1));
    E.order.insert(E.order.end(), huge.begin(), huge.end());
    E.order.insert(E.order.end(), lng.begin(), lng.end());
    E.order.insert(E.order.end(), shrt.begin(), shrt.end());
    const size_t ns = shrt.size(), chunks = (ns + 31) / 32;
    E.chunk.assign(std::max<size_t>(chunks, 1), 0);
    E.len.assign(std::max<size_t>(ns, 1), 0);
    int64_t off = 0;
    for (size_t k = 0; k < chunks; ++k) {
        int64_t L = 0;
        for (size_t j = 32 * k; j < std::min(ns, 32 * k + 32); ++j) {
            const int64_t d = rp[shrt[j] + 1] - rp[shrt[j]];
            E.len[j] = (uint8_t)d;
            L = std::max(L, d);
        }
        E.chunk[k] = off;
        off += 32 * L;
    }
    E.col.assign((size_t)std::max<int64_t>(off, 1), 0);
    E.val.assign((size_t)std::max<int64_t>(off, 1), 0.0);
    for (size_t j = 0; j < ns; ++j) {
        const int64_t p0 = rp[shrt[j]], base = E.chunk[j / 32] + (int64_t)(j % 32);
        for (int64_t e = 0; e < E.len[j]; ++e) {
            E.col[(size_t)(base + 32 * e)] = col[(size_t)(p0 + e)];
            E.val[(size_t)(base + 32 * e)] = val[(size_t)(p0 + e)];
        }
    }
}

// The pre-pass of every pair over all slots at once: control-variate Taylor
// terms and features (two row passes), prediction, coefficients (one row pass;
// with their exponent and scaled FP32 copy for FP32 integrals); or the scaled
// FP32 copy of v.
cudaError_t prepass(mcx_cvbatch *b, cudaStream_t st) {
    const int64_t S = b->slots;
    const unsigned nb = (unsigned)std::max<int64_t>(1, std::min<int64_t>((S + 255) / 256, 152 * 8));
    if (cv_mode(b)) {
        const CvRowSchedule sch{b->sorder, b->scnt, nullptr};
        const CvSell ell{b->ell_col, b->ell_val, b->ell_chunk, b->ell_len};
        double2 *rec = reinterpret_cast<double2 *>(b->work);
        cudaError_t e = cv_taylor_rows(S, b->srp, b->scol, b->sval, b->v, 0.0, b->t_row, sch, &ell, rec,
                                       b->taylor + 3 * S, b->taylor, b->feat, false, st);
        if (e != cudaSuccess) return e;
        if (b->control == MCX_CV_LEARNED) {
            const mcx_status rc = mcx_mlp_predict(b->net, S, b->feat, b->y, st);
            if (rc != MCX_OK) return rc == MCX_E_OOM ? cudaErrorMemoryAllocation : cudaErrorUnknown;
        }
        if ((e = cv_cubic_rows(S, b->srp, b->scol, b->sval, b->taylor, b->control == MCX_CV_LEARNED ? b->y : nullptr,
                               b->t_row, b->t_row + S, sch, &ell, rec, b->ab, b->h, st)) != cudaSuccess)
            return e;
        if ((e = cudaMemsetAsync(b->vexp, 0, sizeof(uint32_t) * b->n_pair, st)) != cudaSuccess) return e;
        if (b->precision == MCX_FP32) {  // the coefficients' exponent per pair and their scaled FP32 copy
            k_pair_exponent<<<nb, 256, 0, st>>>(S, 2, reinterpret_cast<const double *>(b->ab), b->slot_pair, b->vexp);
            k_pair_coef_f32<<<nb, 256, 0, st>>>(S, b->ab, b->slot_pair, b->vexp, b->abf);
        }
    } else if (b->precision == MCX_FP32) {
        cudaError_t e = cudaMemsetAsync(b->vexp, 0, sizeof(uint32_t) * b->n_pair, st);
        if (e != cudaSuccess) return e;
        k_pair_exponent<<<nb, 256, 0, st>>>(S, 1, b->v, b->slot_pair, b->vexp);
        k_pair_pack<<<nb, 256, 0, st>>>(S, b->v, b->slot_pair, b->vexp, b->vf);
    }
    return cudaGetLastError();
}

void launch_walk(const mcx_cvbatch *b, cudaStream_t st) {
    const bool weighted = b->plan->weighted_rows > 0;
    void *fn = pick_walk(cv_mode(b), b->precision == MCX_FP64, weighted, b->staged);
    void *args[] = {const_cast<WalkParams *>(&b->wp), const_cast<CvbArgs *>(&b->ba)};
    cudaLaunchKernel(fn, dim3((unsigned)(b->sms * b->blocks_per_sm)), dim3(WALK_THREADS), args, 0, st);
}

void launch_finish(const mcx_cvbatch *b, cudaStream_t st) {
    if (b->n_warp_pairs == 0) return;
    const dim3 grid((unsigned)((b->warp_pairs_max_n + 255) / 256), (unsigned)b->n_warp_pairs);
    k_cvb_finish<<<grid, 256, 0, st>>>(b->pairs, b->warp_pairs, cv_mode(b),
                                       !cv_mode(b) && b->precision == MCX_FP32, b->ba, b->plan->status);
}

cudaError_t capture(mcx_cvbatch *b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    b->walk_node = nullptr;
    cudaStream_t cs;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaError_t ep = prepass(b, cs);
        cudaMemsetAsync(b->next_item, 0, sizeof(unsigned int), cs);
        launch_walk(b, cs);
        launch_finish(b, cs);
        e = cudaStreamEndCapture(cs, &b->graph);
        if (e == cudaSuccess && ep != cudaSuccess) e = ep;
    }
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) return e;
    if ((e = cudaGraphInstantiate(&b->exec, b->graph, 0)) != cudaSuccess) return e;
    size_t nn = 0;
    cudaGraphGetNodes(b->graph, nullptr, &nn);
    std::vector<cudaGraphNode_t> nodes(nn);
    cudaGraphGetNodes(b->graph, nodes.data(), &nn);
    const void *wf = pick_walk(cv_mode(b), b->precision == MCX_FP64, b->plan->weighted_rows > 0, b->staged);
    for (auto nd : nodes) {
        cudaGraphNodeType ty;
        cudaGraphNodeGetType(nd, &ty);
        if (ty != cudaGraphNodeTypeKernel) continue;
        cudaKernelNodeParams kp;
        if (cudaGraphKernelNodeGetParams(nd, &kp) == cudaSuccess && kp.func == wf) b->walk_node = nd;
    }
    return b->walk_node ? cudaSuccess : cudaErrorUnknown;
}

cudaError_t run_graph(mcx_cvbatch *b, uint64_t seed, cudaStream_t st) {
    set_round_keys(b->wp, seed);
    void *args[] = {&b->wp, &b->ba};
    cudaKernelNodeParams kp;
    cudaError_t e = cudaGraphKernelNodeGetParams(b->walk_node, &kp);
    if (e != cudaSuccess) return e;
    kp.kernelParams = args;
    kp.extra = nullptr;
    if ((e = cudaGraphExecKernelNodeSetParams(b->exec, b->walk_node, &kp)) != cudaSuccess) return e;
    return cudaGraphLaunch(b->exec, st);
}

std::string signature(const mcx_cvbatch *b) {
    char buf[512];
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp pr;
    cudaGetDeviceProperties(&pr, dev);
    uint64_t paths = 0;
    int warp_pairs = 0;
    for (const auto &p : b->pair_host) {
        paths += p.paths * (uint64_t)p.n;
        warp_pairs += p.paths > LANE_MODE_MAX_PATHS;
    }
    snprintf(buf, sizeof buf, "%s|cvbatch|control=%d|prec=%d|pairs=%d|warp_pairs=%d|states=%lld|paths=%llu|nnz=%lld|w=%d",
             pr.name, b->control, b->precision, b->n_pair, warp_pairs, (long long)b->N, (unsigned long long)paths,
             (long long)b->plan->nnz_off, b->plan->weighted_rows > 0 ? 1 : 0);
    return buf;
}

// Time the walk alone on every 8th item for each (chunk, blocks per SM, staging)
// setting and keep the fastest.  Chunk and staging matter only for warp-layout pairs.
cudaError_t autotune(mcx_cvbatch *b, cudaStream_t st) {
    bool any_warp = false;
    for (const auto &p : b->pair_host) any_warp |= b->paths[p.problem] > LANE_MODE_MAX_PATHS;
    const std::vector<uint32_t> Ls = any_warp ? std::vector<uint32_t>{512, 1024, 2048, 4096}
                                              : std::vector<uint32_t>{2048};
    const std::vector<int> bpss = {2, 3, 4, 6};
    const std::vector<int> stg = any_warp ? std::vector<int>{0, 1} : std::vector<int>{1};
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double best = 1e300;
    uint32_t bL = b->chunk;
    int bb = b->blocks_per_sm;
    bool bs = b->staged;
    cudaError_t e = cudaSuccess;
    for (uint32_t L : Ls) {
        b->chunk = L;
        layout_pairs(b);
        if (partials_needed(b) + 1 > b->part_cap) {  // the full run's partials cover every sample
            if ((e = apply_layout(b, st)) != cudaSuccess) break;
        }
        if ((e = cudaMemcpyAsync(b->pairs, b->pair_host.data(), sizeof(CvbPair) * b->n_pair, cudaMemcpyHostToDevice,
                                 st)) != cudaSuccess)
            break;
        if ((e = upload_items(b, make_items(b, 8), st)) != cudaSuccess) break;
        for (int bc : bpss) {
            for (int s : stg) {
                b->blocks_per_sm = bc;
                b->staged = s != 0;
                float ms = 0.f;
                for (int rep = 0; rep < 2; ++rep) {  // warm, then timed
                    cudaMemsetAsync(b->next_item, 0, sizeof(unsigned int), st);
                    cudaEventRecord(e0, st);
                    launch_walk(b, st);
                    cudaEventRecord(e1, st);
                    if ((e = cudaEventSynchronize(e1)) != cudaSuccess) break;
                    cudaEventElapsedTime(&ms, e0, e1);
                }
                if (e != cudaSuccess) break;
                if (ms < best) {
                    best = ms;
                    bL = L;
                    bb = bc;
                    bs = s != 0;
                }
            }
            if (e != cudaSuccess) break;
        }
        if (e != cudaSuccess) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->chunk = bL;
    b->blocks_per_sm = bb;
    b->staged = bs;
    b->tuned_ms = best < 1e300 ? best : 0.0;
    return e;
}

}  // namespace

extern "C" {

mcx_status mcx_cvbatch_create(int32_t count, const mcx_cv_problem *pr, int control, const mcx_mlp *net,
                              int precision, const char *tune_cache, void *stream, mcx_cvbatch **out) {
    NvtxRange nvtx("mcx_cvbatch_create");
    if (!out) return MCX_E_INVALID;
    *out = nullptr;
    if (count < 1 || !pr) return MCX_E_INVALID;
    if (control != MCX_CV_NONE && control != MCX_CV_TAYLOR && control != MCX_CV_LEARNED) return MCX_E_INVALID;
    if (control == MCX_CV_LEARNED && !net) return MCX_E_INVALID;
    if (precision != MCX_FP32 && precision != MCX_FP64) return MCX_E_INVALID;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int64_t N = 0, nnz = 0, slots = 0, snnz = 0;
    std::vector<int64_t> off(count);
    for (int32_t i = 0; i < count; ++i) {
        const mcx_cv_problem &p = pr[i];
        if (p.n < 1 || p.nnz < 0 || !p.row_ptr || (p.nnz > 0 && (!p.col || !p.val)) || p.n_rhs < 1 || !p.v ||
            !p.t || p.paths < 1 || p.paths > (1ull << 40))
            return MCX_E_INVALID;
        if (p.row_ptr[0] != 0 || p.row_ptr[p.n] != p.nnz) return MCX_E_INVALID;
        for (int32_t r = 0; r < p.n_rhs; ++r)
            if (!(p.t[r] > 0.0) || !isfinite(p.t[r])) return MCX_E_INVALID;
        for (int64_t q = 0; q < p.nnz; ++q)
            if (p.col[q] < 0 || p.col[q] >= p.n) return MCX_E_INVALID;
        off[i] = N;
        N += (p.n + CVB_BLOCK - 1) / CVB_BLOCK * CVB_BLOCK;
        nnz += p.nnz;
        slots += p.n * p.n_rhs;
        snnz += p.nnz * p.n_rhs;
    }
    // states of the block-diagonal plan and slots of the pre-pass are indexed in 32 bits
    if (N >= (int64_t)0x7fffffff || slots >= (int64_t)0x7fffffff) return MCX_E_INVALID;
    mcx_cvbatch *b = new (std::nothrow) mcx_cvbatch();
    if (!b) return MCX_E_OOM;
    b->problems = count;
    b->control = control;
    b->precision = precision;
    b->net = net;
    b->N = N;
    b->slots = slots;
    const bool cv = control != MCX_CV_NONE;
    // block-diagonal CSR (host), the pairs, the slot CSR of the pre-pass
    std::vector<int64_t> rp(N + 1, 0);
    std::vector<int32_t> col((size_t)std::max<int64_t>(nnz, 1));
    std::vector<double> val((size_t)std::max<int64_t>(nnz, 1));
    std::vector<double> vall((size_t)std::max<int64_t>(slots, 1));
    std::vector<int32_t> spair((size_t)std::max<int64_t>(slots, 1));
    std::vector<double> trow((size_t)std::max<int64_t>(2 * slots, 1));
    std::vector<int64_t> srp;
    std::vector<int32_t> scol;
    std::vector<double> sval;
    if (cv) {
        srp.assign((size_t)slots + 1, 0);
        scol.resize((size_t)std::max<int64_t>(snnz, 1));
        sval.resize((size_t)std::max<int64_t>(snnz, 1));
    }
    int64_t w = 0, slot = 0, sw = 0;
    for (int32_t i = 0; i < count; ++i) {
        const mcx_cv_problem &p = pr[i];
        double lam = 0.0;  // mean jump rate (cost model)
        for (int64_t r = 0; r < p.n; ++r) {
            rp[off[i] + r] = w;
            for (int64_t q = p.row_ptr[r]; q < p.row_ptr[r + 1]; ++q) {
                col[w] = (int32_t)(p.col[q] + off[i]);
                val[w] = p.val[q];
                if (p.col[q] != r && p.val[q] > 0.0) lam += p.val[q];
                ++w;
            }
        }
        lam /= (double)p.n;
        const int64_t end = (i + 1 < count) ? off[i + 1] : N;
        for (int64_t r = off[i] + p.n; r < end; ++r) rp[r] = w;
        b->paths.push_back(p.paths);
        for (int32_t r = 0; r < p.n_rhs; ++r) {
            CvbPair q{};
            q.off = off[i];
            q.n = p.n;
            q.slot = slot;
            q.paths = p.paths;
            q.path_base = (uint64_t)b->pair_host.size() << 40;
            q.t = p.t[r];
            q.t32 = (float)p.t[r];
            q.problem = i;
            q.rhs = r;
            memcpy(vall.data() + slot, p.v + (size_t)r * (size_t)p.n, sizeof(double) * (size_t)p.n);
            for (int64_t j = 0; j < p.n; ++j) {
                spair[slot + j] = (int32_t)b->pair_host.size();
                trow[slot + j] = p.t[r];
                trow[slots + slot + j] = 1.0 / (p.t[r] * p.t[r] * p.t[r]);
            }
            if (cv)
                for (int64_t j = 0; j < p.n; ++j) {  // this pair's copy of the rows, columns in its slots
                    srp[slot + j] = sw;
                    for (int64_t q2 = p.row_ptr[j]; q2 < p.row_ptr[j + 1]; ++q2) {
                        scol[sw] = (int32_t)(slot + p.col[q2]);
                        sval[sw] = p.val[q2];
                        ++sw;
                    }
                }
            b->pair_host.push_back(q);
            b->cost_per_path.push_back(1.0 + p.t[r] * lam);
            slot += p.n;
        }
    }
    rp[N] = w;
    if (cv) srp[slots] = sw;
    HostEll ell;
    if (cv) build_ell(slots, srp, scol, sval, ell);
    b->n_pair = (int32_t)b->pair_host.size();
    mcx_status rc = mcx_plan_create(N, w, rp.data(), col.data(), val.data(), MCX_PLAN_HOST_INPUT, stream, &b->plan);
    if (rc != MCX_OK) {
        b->plan = nullptr;
        free_cvbatch(b);
        return rc;
    }
    cudaError_t e = cudaSuccess;
    const size_t sl = (size_t)std::max<int64_t>(slots, 1);
    do {
        if ((e = dev_malloc(reinterpret_cast<void **>(&b->v), sizeof(double) * sl)) != cudaSuccess) break;
        if ((e = dev_malloc(reinterpret_cast<void **>(&b->slot_pair), sizeof(int32_t) * sl)) != cudaSuccess) break;
        if ((e = dev_malloc(reinterpret_cast<void **>(&b->mean), sizeof(double) * sl)) != cudaSuccess) break;
        if ((e = dev_malloc(reinterpret_cast<void **>(&b->sem), sizeof(double) * sl)) != cudaSuccess) break;
        if ((e = dev_malloc(reinterpret_cast<void **>(&b->pairs), sizeof(CvbPair) * b->n_pair)) != cudaSuccess) break;
        if ((e = dev_malloc(reinterpret_cast<void **>(&b->warp_pairs), sizeof(int32_t) * b->n_pair)) != cudaSuccess)
            break;
        if ((e = dev_malloc(reinterpret_cast<void **>(&b->vexp), sizeof(uint32_t) * b->n_pair)) != cudaSuccess) break;
        if ((e = dev_malloc(reinterpret_cast<void **>(&b->next_item), 16)) != cudaSuccess) break;
        if (cv) {
            if ((e = dev_malloc(reinterpret_cast<void **>(&b->srp), sizeof(int64_t) * srp.size())) != cudaSuccess) break;
            if ((e = dev_malloc(reinterpret_cast<void **>(&b->scol), sizeof(int32_t) * scol.size())) != cudaSuccess)
                break;
            if ((e = dev_malloc(reinterpret_cast<void **>(&b->sval), sizeof(double) * sval.size())) != cudaSuccess)
                break;
            if ((e = dev_malloc(reinterpret_cast<void **>(&b->t_row), sizeof(double) * trow.size())) != cudaSuccess)
                break;
            if ((e = dev_malloc(reinterpret_cast<void **>(&b->taylor), 4 * sizeof(double) * sl)) != cudaSuccess) break;
            if ((e = dev_malloc(reinterpret_cast<void **>(&b->feat), 5 * sizeof(float) * sl)) != cudaSuccess) break;
            if ((e = dev_malloc(reinterpret_cast<void **>(&b->y), sizeof(float) * sl)) != cudaSuccess) break;
            if ((e = dev_malloc(reinterpret_cast<void **>(&b->ab), sizeof(double2) * sl)) != cudaSuccess) break;
            if ((e = dev_malloc(reinterpret_cast<void **>(&b->h), sizeof(double) * sl)) != cudaSuccess) break;
            if ((e = dev_malloc(reinterpret_cast<void **>(&b->work), sizeof(double2) * sl)) != cudaSuccess) break;
            if ((e = dev_malloc(reinterpret_cast<void **>(&b->sorder), sizeof(int32_t) * sl)) != cudaSuccess) break;
            if ((e = dev_malloc(reinterpret_cast<void **>(&b->scnt), sizeof(uint32_t) * CV_ROW_CNT)) != cudaSuccess)
                break;
            if ((e = dev_malloc(reinterpret_cast<void **>(&b->ell_col), sizeof(int32_t) * ell.col.size())) !=
                cudaSuccess)
                break;
            if ((e = dev_malloc(reinterpret_cast<void **>(&b->ell_val), sizeof(double) * ell.val.size())) !=
                cudaSuccess)
                break;
            if ((e = dev_malloc(reinterpret_cast<void **>(&b->ell_chunk), sizeof(int64_t) * ell.chunk.size())) !=
                cudaSuccess)
                break;
            if ((e = dev_malloc(reinterpret_cast<void **>(&b->ell_len), ell.len.size())) != cudaSuccess) break;
            if (precision == MCX_FP32 &&
                (e = dev_malloc(reinterpret_cast<void **>(&b->abf), sizeof(float2) * sl)) != cudaSuccess)
                break;
        } else {
            if ((e = dev_malloc(reinterpret_cast<void **>(&b->vf), sizeof(float) * sl)) != cudaSuccess) break;
        }
        cudaMemsetAsync(b->vexp, 0, sizeof(uint32_t) * b->n_pair, st);
        if (cv) {
            cudaMemcpyAsync(b->srp, srp.data(), sizeof(int64_t) * srp.size(), cudaMemcpyHostToDevice, st);
            cudaMemcpyAsync(b->scol, scol.data(), sizeof(int32_t) * scol.size(), cudaMemcpyHostToDevice, st);
            cudaMemcpyAsync(b->sval, sval.data(), sizeof(double) * sval.size(), cudaMemcpyHostToDevice, st);
            cudaMemcpyAsync(b->t_row, trow.data(), sizeof(double) * trow.size(), cudaMemcpyHostToDevice, st);
            cudaMemcpyAsync(b->sorder, ell.order.data(), sizeof(int32_t) * ell.order.size(), cudaMemcpyHostToDevice, st);
            cudaMemcpyAsync(b->scnt, ell.cnt, sizeof(ell.cnt), cudaMemcpyHostToDevice, st);
            cudaMemcpyAsync(b->ell_col, ell.col.data(), sizeof(int32_t) * ell.col.size(), cudaMemcpyHostToDevice, st);
            cudaMemcpyAsync(b->ell_val, ell.val.data(), sizeof(double) * ell.val.size(), cudaMemcpyHostToDevice, st);
            cudaMemcpyAsync(b->ell_chunk, ell.chunk.data(), sizeof(int64_t) * ell.chunk.size(),
                            cudaMemcpyHostToDevice, st);
            cudaMemcpyAsync(b->ell_len, ell.len.data(), ell.len.size(), cudaMemcpyHostToDevice, st);
        }
        cudaMemcpyAsync(b->slot_pair, spair.data(), sizeof(int32_t) * sl, cudaMemcpyHostToDevice, st);
        if ((e = cudaMemcpyAsync(b->v, vall.data(), sizeof(double) * sl, cudaMemcpyHostToDevice, st)) != cudaSuccess)
            break;
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
        WalkParams &wp = b->wp;
        wp.node = b->plan->node;
        wp.node64 = b->plan->node64;
        wp.edge_col = b->plan->edge_col;
        wp.edge16 = b->plan->edge16;
        wp.nsteps = 1;
        wp.n = N;
        wp.max_events = 1u << 30;
        wp.status = b->plan->status;
        CvbArgs &ba = b->ba;
        ba.pairs = b->pairs;
        ba.next_item = b->next_item;
        ba.ab = b->ab;
        ba.h = b->h;
        ba.abf = b->abf;
        ba.v = b->v;
        ba.vf = b->vf;
        ba.vexp = b->vexp;
        ba.mean = b->mean;
        ba.sem = b->sem;
        // one pre-pass outside the graph, so the autotuner's walks read real coefficients
        if ((e = prepass(b, st)) != cudaSuccess) break;
        // schedule: cached, else autotuned
        const std::string key = signature(b);
        long L = 0, k = 0, s = 1;
        if (tune_cache_get(tune_cache, key, "chunk", &L) && tune_cache_get(tune_cache, key, "blocks_per_sm", &k) &&
            L > 0 && k > 0) {
            tune_cache_get(tune_cache, key, "staged", &s);
            b->chunk = (uint32_t)L;
            b->blocks_per_sm = (int)k;
            b->staged = s != 0;
        } else {
            set_round_keys(b->wp, 0x5eed);
            if ((e = autotune(b, st)) != cudaSuccess) break;
            tune_cache_put(tune_cache, key,
                           {{"chunk", (long)b->chunk}, {"blocks_per_sm", (long)b->blocks_per_sm},
                            {"staged", b->staged ? 1L : 0L}},
                           b->tuned_ms);
        }
        if ((e = apply_layout(b, st)) != cudaSuccess) break;
        if ((e = capture(b)) != cudaSuccess) break;
        cudaMemsetAsync(b->plan->status, 0, 4 * STATUS_SYNC_WORDS, st);  // the tuning runs' statistics
        e = cudaStreamSynchronize(st);
    } while (0);
    if (e != cudaSuccess) {
        cudaStreamSynchronize(st);
        free_cvbatch(b);
        return cvb_status(e);
    }
    *out = b;
    return MCX_OK;
}

mcx_status mcx_cvbatch_set_paths(mcx_cvbatch *b, const uint64_t *paths, void *stream) {
    NvtxRange nvtx("mcx_cvbatch_set_paths");
    if (!b || !paths) return MCX_E_INVALID;
    for (int32_t i = 0; i < b->problems; ++i)
        if (paths[i] < 1 || paths[i] > (1ull << 40)) return MCX_E_INVALID;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaStreamSynchronize(st);  // no run of the old layout in flight
    if (e != cudaSuccess) return cvb_status(e);
    for (int32_t i = 0; i < b->problems; ++i) b->paths[i] = paths[i];
    if ((e = apply_layout(b, st)) != cudaSuccess) return cvb_status(e);
    if ((e = capture(b)) != cudaSuccess) return cvb_status(e);
    return cvb_status(cudaStreamSynchronize(st));
}

mcx_status mcx_cvbatch_run(mcx_cvbatch *b, uint64_t seed, void *stream) {
    NvtxRange nvtx("mcx_cvbatch_run");
    if (!b) return MCX_E_INVALID;
    return cvb_status(run_graph(b, seed, static_cast<cudaStream_t>(stream)));
}

mcx_status mcx_cvbatch_result(const mcx_cvbatch *b, int32_t problem, int32_t rhs, double *x, double *sem,
                              void *stream) {
    if (!b || !x) return MCX_E_INVALID;
    for (const auto &p : b->pair_host) {
        if (p.problem != problem || p.rhs != rhs) continue;
        cudaStream_t st = static_cast<cudaStream_t>(stream);
        cudaError_t e = cudaMemcpyAsync(x, b->mean + p.slot, sizeof(double) * p.n, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess && sem)
            e = cudaMemcpyAsync(sem, b->sem + p.slot, sizeof(double) * p.n, cudaMemcpyDeviceToDevice, st);
        return cvb_status(e);
    }
    return MCX_E_INVALID;
}

mcx_status mcx_cvbatch_coefficients(const mcx_cvbatch *b, int32_t problem, int32_t rhs, double *coef,
                                    void *stream) {
    if (!b || !coef || !cv_mode(b)) return MCX_E_INVALID;
    for (const auto &p : b->pair_host) {
        if (p.problem != problem || p.rhs != rhs) continue;
        const cudaStream_t st = static_cast<cudaStream_t>(stream);
        const cudaError_t e = cudaMemcpyAsync(coef, b->ab + p.slot, sizeof(double2) * (size_t)p.n,
                                              cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return cvb_status(e);
        return cvb_status(cudaMemcpyAsync(coef + 2 * p.n, b->h + p.slot, sizeof(double) * (size_t)p.n,
                                          cudaMemcpyDeviceToDevice, st));
    }
    return MCX_E_INVALID;
}

mcx_status mcx_cvbatch_get_info(const mcx_cvbatch *b, mcx_cvbatch_info *info) {
    if (!b || !info) return MCX_E_INVALID;
    info->problems = b->problems;
    info->pairs = b->n_pair;
    info->states = b->N;
    uint64_t total = 0;
    for (const auto &p : b->pair_host) total += p.paths * (uint64_t)p.n;
    info->total_paths = total;
    info->work_items = b->n_items;
    info->chunk = b->chunk;
    info->blocks_per_sm = b->blocks_per_sm;
    info->grid = b->sms * b->blocks_per_sm;
    info->staged = b->staged ? 1 : 0;
    info->control = b->control;
    info->tuned_ms = b->tuned_ms;
    return MCX_OK;
}

mcx_status mcx_cvbatch_sync(mcx_cvbatch *b, void *stream, mcx_stats *stats) {
    if (!b) return MCX_E_INVALID;
    mcx_status rc = mcx_sync(b->plan, stream, stats);
    if (rc == MCX_OK && b->control == MCX_CV_LEARNED) rc = mcx_mlp_sync(const_cast<mcx_mlp *>(b->net), stream);
    return rc;
}

void mcx_cvbatch_destroy(mcx_cvbatch *b) {
    if (!b) return;
    cudaDeviceSynchronize();
    free_cvbatch(b);
}

}  // extern "C"
