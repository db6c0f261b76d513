// Double-float arithmetic: a value is the unevaluated sum h + l of two FP32
// numbers (about 48 significant bits).  GB300 runs FP64 at a small fraction
// of its FP32 rate, so the per-edge sums of the node features accumulate here
// on the FP32 pipe.  (Sparse products keep FP64: splitting each FP64 operand
// costs more integer work than the FP64 multiply-add it would replace.)  Products use the exact FMA residual
// (Dekker's product with a fused multiply-add); sums use Knuth's TwoSum
// (Knuth, TAOCP vol. 2, 4.2.2).  FP64 inputs are split into (h, l) with
// integer operations only (no FP64 instruction per element).
#pragma once

#include <stdint.h>

namespace mcx {

struct df {
    float h, l;
};

// Split a finite double d into h + l: h is d with its significand truncated
// to 24 bits (integer bit manipulation), l = d - h exactly before the
// conversion of the 29 dropped bits to FP32 (which keeps 24 of them).  Exact
// to about 2^-47 relative.  Needs 2^-74 <= |d| < 2^127 (zero is exact); other
// inputs set *bad and return an unspecified value.
__device__ __forceinline__ df df_split(double d, bool &bad) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(d);
    const uint32_t hi = (uint32_t)(b >> 32), lo = (uint32_t)b;
    const int e = (int)((hi >> 20) & 0x7ffu) - 1023;
    if ((b << 1) == 0ull) return df{0.0f, 0.0f};
    if (e < -74 || e > 127) bad = true;
    const uint32_t sign = hi & 0x80000000u;
    const float h = __uint_as_float(sign | ((uint32_t)(e + 127) << 23) | ((hi & 0x000fffffu) << 3) | (lo >> 29));
    const float scale = __uint_as_float((uint32_t)(e - 52 + 127) << 23);  // 2^(e-52), normal for e >= -74
    const float l = __fmul_rn(__uint2float_rn(lo & 0x1fffffffu), scale);
    return df{h, __uint_as_float(__float_as_uint(l) | sign)};
}

__device__ __forceinline__ double df_to_double(df a) { return (double)a.h + (double)a.l; }

// a * b, not renormalised: h = fl(ah bh), l = the exact residual of that
// product plus the cross terms ah bl + al bh (al bl is below 2^-48).
__device__ __forceinline__ df df_mul(df a, df b) {
    const float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);
    e = __fmaf_rn(a.h, b.l, e);
    e = __fmaf_rn(a.l, b.h, e);
    return df{p, e};
}

// s + a: TwoSum of the high parts, low parts added to the error.
__device__ __forceinline__ df df_add(df s, df a) {
    const float t = __fadd_rn(s.h, a.h);
    const float bp = __fsub_rn(t, s.h);
    const float err = __fadd_rn(__fsub_rn(s.h, __fsub_rn(t, bp)), __fsub_rn(a.h, bp));
    return df{t, __fadd_rn(__fadd_rn(s.l, a.l), err)};
}

// Renormalise so that |l| <= ulp(h)/2 (Fast2Sum).
__device__ __forceinline__ df df_norm(df a) {
    const float h = __fadd_rn(a.h, a.l);
    return df{h, __fsub_rn(a.l, __fsub_rn(h, a.h))};
}

__device__ __forceinline__ df df_shfl_xor(df a, int o) {
    return df{__shfl_xor_sync(0xffffffffu, a.h, o), __shfl_xor_sync(0xffffffffu, a.l, o)};
}

}  // namespace mcx
