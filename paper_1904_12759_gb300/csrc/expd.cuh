// FP64 exponential of an FP32 argument for the control-variate coefficients
// (xhat = T2 e^y, y the network's FP32 output), by Tang's table-driven method
// (P. T. P. Tang, ACM TOMS 15(2), 1989): y = (64 m + j) ln(2)/64 + r with
// |r| <= ln(2)/128 (plus rounding), e^y = 2^m 2^(j/64) e^r, e^r - 1 from its
// Taylor series to r^6 (the next term is below 2^-60).  The reduction is exact
// (N ln(2)/64 = N L1 + N L2, N L1 exact for |N| < 2^17), so the result is
// within about one unit in the last place of e^y.  About a dozen FP64
// operations, a third of a general-purpose double exponential: GB300 runs FP64
// at a small fraction of its FP32 rate.  Arguments with |y| >= 700 (and
// non-finite ones) take the library's exp.
#pragma once

#include <math.h>
#include <stdint.h>

#include "exp_table.cuh"

namespace mcx {

__device__ __forceinline__ double exp_of_f32(float y) {
    if (!(fabsf(y) < 700.0f)) return exp((double)y);
    const int N = (int)rintf(__fmul_rn(y, 92.33248261689366f));  // about y 64/ln(2)
    const double Nd = (double)N;
    double r = __fma_rn(-Nd, EXP_L1, (double)y);  // exact
    r = __fma_rn(-Nd, EXP_L2, r);
    double p = __fma_rn(r, 1.0 / 720.0, 1.0 / 120.0);
    p = __fma_rn(p, r, 1.0 / 24.0);
    p = __fma_rn(p, r, 1.0 / 6.0);
    p = __fma_rn(p, r, 0.5);
    p = __fma_rn(p, r, 1.0);
    p = __dmul_rn(p, r);  // e^r - 1
    const double T = __longlong_as_double((long long)c_exp_table[N & 63]);
    const int m = N >> 6;  // N = 64 m + (N & 63); |m| <= 1010: 2^m is a normal FP64 number
    return __dmul_rn(__fma_rn(T, p, T), __longlong_as_double((long long)(m + 1023) << 52));
}

}  // namespace mcx
