// Residual integral of the control-variate walkers (variance reduction,
// Sec. 5): over a hold of length D in state j, starting with remaining time r,
// the integral of R(r - u) e^{delta_j u} du for R(tau) = a tau^2 + b tau^3,
// written as sum_k c_k D^{k+1} phi_k(delta_j D) with phi_k(z) = int_0^1 e^{zs}
// s^k ds (series for small |z|, the recursion phi_k = (e^z - k phi_{k-1})/z
// otherwise).  Used by the single-problem (cv.cu) and batched (cvbatch.cu)
// control-variate walkers.
#pragma once

#include <math.h>

#include "mcx_internal.cuh"

namespace mcx {
namespace {

// phi_k(z) = sum_n z^n / (n! (n + k + 1)): Horner coefficients 1/(n! (n+k+1)).
struct PhiSeries {
    float c[4][11];  // FP32: 11 terms for |z| <= 1 (remainder below 2e-9)
};
__host__ __device__ constexpr PhiSeries phi_series() {
    PhiSeries s{};
    for (int k = 0; k < 4; ++k) {
        double f = 1.0;  // n!
        for (int n = 0; n < 11; ++n) {
            if (n > 0) f *= n;
            s.c[k][n] = (float)(1.0 / (f * (n + k + 1)));
        }
    }
    return s;
}
__constant__ PhiSeries c_phi = phi_series();

template <typename R>
__device__ __forceinline__ void phis(R z, R ph[4]) {
    if (sizeof(R) == 4) {
        if (fabsf((float)z) <= 1.0f) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                float p = c_phi.c[k][10];
#pragma unroll
                for (int n = 9; n >= 0; --n) p = fmaf(p, (float)z, c_phi.c[k][n]);
                ph[k] = (R)p;
            }
        } else {
            const float ez = expf((float)z), iz = 1.0f / (float)z;
            ph[0] = (R)((ez - 1.0f) * iz);
            ph[1] = (R)((ez - (float)ph[0]) * iz);
            ph[2] = (R)((ez - 2.0f * (float)ph[1]) * iz);
            ph[3] = (R)((ez - 3.0f * (float)ph[2]) * iz);
        }
        return;
    }
    // FP64: series to 40 terms for |z| <= 2, else the recursion
    if (fabs((double)z) <= 2.0) {
        R term = (R)1, s0 = 0, s1 = 0, s2 = 0, s3 = 0;
        for (int n = 0; n < 40; ++n) {
            s0 += term / (R)(n + 1);
            s1 += term / (R)(n + 2);
            s2 += term / (R)(n + 3);
            s3 += term / (R)(n + 4);
            term *= z / (R)(n + 1);
        }
        ph[0] = s0; ph[1] = s1; ph[2] = s2; ph[3] = s3;
    } else {
        const R ez = (R)exp((double)z);
        ph[0] = (ez - (R)1) / z;
        ph[1] = (ez - (R)1 * ph[0]) / z;
        ph[2] = (ez - (R)2 * ph[1]) / z;
        ph[3] = (ez - (R)3 * ph[2]) / z;
    }
}

template <typename R>
__device__ __forceinline__ R hold_integral(R a, R b, R delta, R r, R D) {
    const R c0 = a * r * r + b * r * r * r;
    const R c1 = (R)-2 * a * r - (R)3 * b * r * r;
    const R c2 = a + (R)3 * b * r;
    const R c3 = -b;
    R ph[4];
    phis<R>(delta * D, ph);
    return c0 * D * ph[0] + c1 * D * D * ph[1] + c2 * D * D * D * ph[2] + c3 * D * D * D * D * ph[3];
}

// FP32 residual integrals read the coefficient pairs (a_j, b_j) as an FP32 copy
// scaled by 2^-k, k the binary exponent of the largest |a|, |b| (from the
// biased word; the scaling is exact, the copy rounds once): one 8-byte load per
// hold and no FP64 arithmetic in the walk, with the residuals and their squares
// inside the FP32 range whatever the scale of v.  Results are scaled back by 2^k.
__global__ void k_coef_f32(int64_t n, const double2 *__restrict__ ab, const uint32_t *__restrict__ word,
                           float2 *__restrict__ out) {
    const uint32_t e = *word;
    const int k = e ? (int)e - (int)VEXP_BIAS : 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double2 c = ab[i];
        out[i] = make_float2(__double2float_rn(ldexp(c.x, -k)), __double2float_rn(ldexp(c.y, -k)));
    }
}

}  // namespace
}  // namespace mcx
