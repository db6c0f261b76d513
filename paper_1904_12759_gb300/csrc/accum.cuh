// Per-path weight accumulators of the walkers and their merges: lanes keep
// log-shifted sums of w = e^{logW} v and w^2 (FP32 compensated or FP64), warps
// merge them by log-sum-exp, and finish_entry turns shifted sums into a mean
// and a standard error.
#pragma once

#include <math.h>

#include "mcx_internal.cuh"

namespace mcx {
namespace {

// ---------------------------------------------------------------------------
// Lane accumulators and their warp merges (result in lane 0).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void kahan_add(float &s, float &c, float x) {
    const float y = __fsub_rn(x, c);
    const float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
}

// (h, l) += (h2, l2) for unevaluated float pairs: TwoSum of the high parts, then renormalise.
__device__ __forceinline__ void pair_add(float &h, float &l, float h2, float l2) {
    const float s = __fadd_rn(h, h2);
    const float bp = __fsub_rn(s, h);
    const float e = __fadd_rn(__fsub_rn(h, __fsub_rn(s, bp)), __fsub_rn(h2, bp));
    const float lo = __fadd_rn(__fadd_rn(l, l2), e);
    h = __fadd_rn(s, lo);
    l = __fsub_rn(lo, __fsub_rn(h, s));
}

// Sum of w: compensated (it is the estimate).  Sum of w^2: plain FP32 fma
// (it only feeds the standard error; ~31 terms per lane keep it within 1e-5).
struct Acc32 {
    float m = -INFINITY, s1 = 0.f, c1 = 0.f, s2 = 0.f, c2 = 0.f;
    __device__ __forceinline__ void add(float L, float v) {
        if (!(L <= m + 8.0f)) {  // first path, a new larger weight, or a non-finite one
            const float sc = (m == -INFINITY) ? 0.0f : expf(m - L);
            s1 *= sc; c1 *= sc; s2 *= sc * sc;
            m = L;
        }
        const float wv = __fmul_rn(expf(__fsub_rn(L, m)), v);
        kahan_add(s1, c1, wv);
        s2 = __fmaf_rn(wv, wv, s2);
    }
    __device__ __forceinline__ void lane_result(double &S1, double &S2, double &Mw) const {
        S1 = (double)s1 - (double)c1;
        S2 = (double)s2;
        Mw = (double)m;
    }
    __device__ __forceinline__ void warp_merge(double &S1, double &S2, double &Mw) const {
        float mw = m;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mw = fmaxf(mw, __shfl_xor_sync(0xffffffffu, mw, o));
        const float sc = (m == -INFINITY) ? 0.0f : expf(__fsub_rn(m, mw));
        const float sc2 = __fmul_rn(sc, sc);
        float h1 = __fmul_rn(s1, sc), l1 = __fmul_rn(-c1, sc);
        float h2 = __fmul_rn(s2, sc2), l2 = __fmul_rn(-c2, sc2);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            pair_add(h1, l1, __shfl_xor_sync(0xffffffffu, h1, o), __shfl_xor_sync(0xffffffffu, l1, o));
            pair_add(h2, l2, __shfl_xor_sync(0xffffffffu, h2, o), __shfl_xor_sync(0xffffffffu, l2, o));
        }
        S1 = (double)h1 + (double)l1;
        S2 = (double)h2 + (double)l2;
        Mw = (double)mw;
    }
};

__device__ __forceinline__ double warp_max(double x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_xor_sync(0xffffffffu, x, o));
    return x;
}
__device__ __forceinline__ double warp_sum(double x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

struct Acc64 {
    double m = -INFINITY, s1 = 0.0, s2 = 0.0;
    __device__ __forceinline__ void add(double L, double v) {
        if (!(L <= m + 64.0)) {
            const double sc = (m == -INFINITY) ? 0.0 : exp(m - L);
            s1 *= sc; s2 *= sc * sc;
            m = L;
        }
        const double wv = __dmul_rn(exp(__dsub_rn(L, m)), v);
        s1 = __dadd_rn(s1, wv);
        s2 = __fma_rn(wv, wv, s2);
    }
    __device__ __forceinline__ void lane_result(double &S1, double &S2, double &Mw) const {
        S1 = s1;
        S2 = s2;
        Mw = m;
    }
    __device__ __forceinline__ void warp_merge(double &S1, double &S2, double &Mw) const {
        const double mw = warp_max(m);
        const double sc = (m == -INFINITY) ? 0.0 : exp(m - mw);
        S1 = warp_sum(sc * s1);
        S2 = warp_sum(sc * sc * s2);
        Mw = mw;
    }
};

// mean and standard error from shifted sums over M paths, times vs (the power
// of two the FP32 copy of v was scaled by, 1 for FP64 paths)
__device__ __forceinline__ void finish_entry(double s1, double s2, double m, double M, double vs, double *mean,
                                             double *sem, uint32_t *status) {
    const double scale = exp(m);
    const double mu = s1 / M;
    double var = M > 1.0 ? (s2 - s1 * mu) / (M - 1.0) : 0.0;
    if (var < 0.0) var = 0.0;
    const double mv = scale * mu * vs;
    const double se = scale * sqrt(var / M) * vs;
    *mean = mv;
    if (sem) *sem = se;
    if (!isfinite(mv) || !isfinite(se)) atomicOr(status, ST_OVERFLOW);
}

}  // namespace
}  // namespace mcx
