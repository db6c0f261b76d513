// Internal definitions of the mcx library: the plan, the packed node and edge
// records the walkers gather, and the device primitives of the draw schedule
// (Philox4x32-10, uniform maps, logarithms).
//
// Every floating-point step that decides a path (holding time, remaining
// time, grid counts, log-weight) is written with explicit round-to-nearest
// intrinsics (__fadd_rn, __fmul_rn, __fmaf_rn, and the double versions), and
// the library is compiled with --fmad=false, so no contraction or
// reassociation can change a path.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/mcx.h"
#include "ln_table.cuh"

namespace mcx {

// ---------------------------------------------------------------------------
// Packed records.
//
// One 32-byte node record per row (one DRAM/L2 sector per gather): the CSR
// offset of the row's kept off-diagonal entries, their count, the FP32 rate
// reciprocal and potential, and the row's v value in FP32 (written per
// estimate so that the end-of-path read of v costs nothing extra).
// ---------------------------------------------------------------------------
struct __align__(32) NodeRec {
    int64_t row_start;  // offset into the edge arrays
    int32_t deg;        // kept off-diagonal entries (a_ij > 0, j != i)
    uint32_t flags;     // bit 0: alias-table (weighted) row
    float inv_rate;     // (float)(1 / lambda_i), lambda_i = sum_{j != i} a_ij
    float delta;        // (float)(a_ii + lambda_i), the potential D_ii
    float v;            // (float)v_i of the current estimate
    uint32_t pad;
};
static_assert(sizeof(NodeRec) == 32, "node record must be one 32-byte sector");

// FP64 path version: exact-precision rate reciprocal, potential and v.
struct __align__(32) NodeRec64 {
    double inv_rate;
    double delta;
    double v;
    double pad;
};
static_assert(sizeof(NodeRec64) == 32, "FP64 node record must be one 32-byte sector");

constexpr uint32_t NODE_WEIGHTED = 1u;

// Alias entry of a weighted row: slot k keeps its own column iff w3 < thresh,
// otherwise it jumps to alias_col.
struct __align__(8) AliasEnt {
    int32_t alias_col;
    uint32_t thresh;
};

// Packed edge record of a weighted plan (one 16-byte load per jump): the
// slot's own column, its alias column and the keep-own threshold.  Rows whose
// kept entries are all equal alias themselves (threshold 0xFFFFFFFF).
struct __align__(16) Edge16 {
    int32_t col;
    int32_t alias_col;
    uint32_t thresh;
    uint32_t pad;
};

// Device status bits latched in the plan.
constexpr uint32_t ST_OVERFLOW = 1u;
constexpr uint32_t ST_BAD_STRUCT = 2u;
constexpr uint32_t ST_NEG_OFFDIAG = 4u;
constexpr uint32_t ST_NONFINITE = 8u;
constexpr uint32_t ST_BAD_ENTRY = 16u;
constexpr uint32_t ST_BAD_V = 32u;

// Status words: the first STATUS_SYNC_WORDS are read and cleared by mcx_sync.
constexpr int STATUS_SYNC_WORDS = 8;
constexpr int STATUS_WORDS = 16;
constexpr int STATUS_VEXP = 8;
constexpr int STATUS_CEXP = 9;  // exponent of the control-variate coefficients (see cv.cu)
constexpr uint32_t VEXP_BIAS = 2048u;

// The FP32 node records hold v scaled by a power of two, v * 2^-k with k the
// binary exponent of the largest finite |v_i| (so |v| < 2 there): the per-path
// weights and their squares then stay inside the FP32 range whatever the scale
// of v, and the scaling is exact.  k is kept in status word STATUS_VEXP as
// k + VEXP_BIAS (0 when v has no nonzero finite entry, k = 0); results of FP32
// paths are multiplied by 2^k when they are finished.
__device__ __forceinline__ double v_scale(const uint32_t *status) {
    const uint32_t e = status[STATUS_VEXP];
    return e ? ldexp(1.0, (int)e - (int)VEXP_BIAS) : 1.0;
}

// 2^k for a biased exponent word (0: k = 0).
__device__ __forceinline__ double exp_scale(uint32_t e) { return e ? ldexp(1.0, (int)e - (int)VEXP_BIAS) : 1.0; }

// Largest biased exponent (ilogb + VEXP_BIAS) of the finite nonzero |x_i|,
// i < n, merged into *word by atomicMax (the word is cleared before the launch).
__device__ __forceinline__ void exponent_max(int64_t n, const double *__restrict__ x, uint32_t *word) {
    uint32_t e = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double y = fabs(x[i]);
        if (y > 0.0 && y <= 1.7976931348623157e308) e = max(e, (uint32_t)(ilogb(y) + (int)VEXP_BIAS));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, o));
    if ((threadIdx.x & 31) == 0 && e) atomicMax(word, e);
}

}  // namespace mcx

struct mcx_plan {
    int64_t n = 0;
    int64_t nnz = 0;
    int64_t nnz_off = 0;
    int64_t weighted_rows = 0;
    int32_t max_deg = 0;
    int device = 0;
    mcx::NodeRec *node = nullptr;      // [n]
    mcx::NodeRec64 *node64 = nullptr;  // [n]
    int32_t *edge_col = nullptr;       // [nnz_off]
    mcx::Edge16 *edge16 = nullptr;     // [nnz_off] if weighted_rows > 0 (packed column + alias table)
    uint32_t *status = nullptr;        // device words: [0] status bits, [2..3] paths (u64), [4..5] jumps (u64)
                                       // (cleared by mcx_sync); [8] exponent of the FP32 copy of v (see v_scale)
    void *scratch = nullptr;           // grow-only scratch for chunk partials
    size_t scratch_bytes = 0;
    void *fwd = nullptr;               // forward-form scratch (start tables, deposits), made on first use
    size_t fwd_bytes = 0;
    bool zero_potential = false;       // every delta_i == 0 exactly (forward weights are 1)
    bool fwd_ones = false;             // the forward start tables currently hold v = 1
    int64_t device_bytes = 0;
};

namespace mcx {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds; each round
// multiplies counter words 0 and 2 by the two Philox constants, and mixes the
// high halves with words 1 and 3 and the round key; the key is advanced by
// the two Weyl increments between rounds.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const uint32_t lo0 = 0xD2511F53u * c.x;
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// Uniform in (0, 1] from the top 24 bits (exact in FP32, never 0).
__device__ __forceinline__ float unif24(uint32_t w0) {
    return __fmul_rn(__uint2float_rn(16777216u - (w0 >> 8)), 5.9604644775390625e-8f /* 2^-24 */);
}

// Uniform in (0, 1] from 53 bits of (w0, w1) (exact in FP64, never 0).
__device__ __forceinline__ double unif53(uint32_t w0, uint32_t w1) {
    const unsigned long long m = ((unsigned long long)w0 << 21) | (unsigned long long)(w1 >> 11);
    return __dmul_rn(__ull2double_rn(9007199254740992ull - m), 1.1102230246251565e-16 /* 2^-53 */);
}

// Natural logarithm of a positive normal float, table-driven after Tang
// ("Table-driven implementation of the logarithm function in IEEE
// floating-point arithmetic", ACM TOMS 16(4), 1990), without a division:
//   x = 2^E M, M in [1, 2); j = the breakpoint c_j = 1 + j/64 nearest M
//   (j = 0..64, from the top mantissa bits rounded);
//   r = M (1/c_j) - 1 in one fma, |r| <= 2^-7;
//   ln(1 + r) = r - r^2/2 + r^3/3 - r^4/4 (Taylor, truncation below 2^-37 |r|);
//   ln x = e ln2 + L_j + ln(1 + r), with L_j = -ln(1/c_j as rounded) and
//   e = E, or, for j >= 27 (c_j > sqrt2), L_j = -ln(2/c_j as rounded) and
//   e = E + 1, so that L_j stays within [-ln sqrt2, ln sqrt2] and nothing
//   cancels near x = 1.  Within 2 ulp of the correctly rounded logarithm.
__device__ __forceinline__ float ln_f32(float x) {
    const uint32_t b = __float_as_uint(x);
    const uint32_t mb = b & 0x007fffffu;
    const int j = (int)((mb + 0x10000u) >> 17);
    const int e = (int)(b >> 23) - 127 + (j >= LN_TABLE_BINADE_SPLIT ? 1 : 0);
    const uint2 row = __ldg(&c_ln_table[j]);
    const float r = __fmaf_rn(__uint_as_float(mb | 0x3f800000u), __uint_as_float(row.x), -1.0f);
    float q = __fmaf_rn(r, -0.25f, 1.0f / 3.0f);
    q = __fmaf_rn(q, r, -0.5f);
    const float p = __fmaf_rn(__fmul_rn(r, r), q, r);
    return __fadd_rn(__fmaf_rn(__int2float_rn(e), 0.693147181f, __uint_as_float(row.y)), p);
}

// Same construction in FP64 with the series carried to z^11/25.
__device__ __forceinline__ double ln_f64(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    int e = (int)((b >> 52) & 0x7ffull) - 1023;
    double m = __longlong_as_double((long long)((b & 0x000fffffffffffffull) | 0x3ff0000000000000ull));
    if (m > 1.4142135623730951) {
        m = __dmul_rn(m, 0.5);
        e = e + 1;
    }
    const double s = __ddiv_rn(__dsub_rn(m, 1.0), __dadd_rn(m, 1.0));
    const double z = __dmul_rn(s, s);
    double q = 1.0 / 25.0;
    q = __fma_rn(q, z, 1.0 / 23.0);
    q = __fma_rn(q, z, 1.0 / 21.0);
    q = __fma_rn(q, z, 1.0 / 19.0);
    q = __fma_rn(q, z, 1.0 / 17.0);
    q = __fma_rn(q, z, 1.0 / 15.0);
    q = __fma_rn(q, z, 1.0 / 13.0);
    q = __fma_rn(q, z, 1.0 / 11.0);
    q = __fma_rn(q, z, 1.0 / 9.0);
    q = __fma_rn(q, z, 1.0 / 7.0);
    q = __fma_rn(q, z, 1.0 / 5.0);
    q = __fma_rn(q, z, 1.0 / 3.0);
    const double s2 = __dadd_rn(s, s);
    const double lnm = __fma_rn(__dmul_rn(s2, z), q, s2);
    return __fma_rn(__int2double_rn(e), 0.6931471805599453, lnm);
}

__device__ __forceinline__ NodeRec load_node(const NodeRec *__restrict__ node, int32_t j) {
    const int4 *p = reinterpret_cast<const int4 *>(node + j);
    const int4 a = __ldg(p);
    const int4 b = __ldg(p + 1);
    NodeRec r;
    r.row_start = ((int64_t)(uint32_t)a.y << 32) | (uint32_t)a.x;
    r.deg = a.z;
    r.flags = (uint32_t)a.w;
    r.inv_rate = __int_as_float(b.x);
    r.delta = __int_as_float(b.y);
    r.v = __int_as_float(b.z);
    r.pad = (uint32_t)b.w;
    return r;
}

// Canonical Vose alias construction for d weights w[0..d) with sum lam (one
// thread, FP64): scaled weights q_k = (w_k d) / lam; indices with q < 1 go to
// the "small" list, the rest to "large", both in index order; pairs are popped
// from the back; the large entry keeps (q_l + q_s) - 1; leftovers alias
// themselves.  out[k] = {id(alias slot), floor(q_k 2^32)}; keep-own-slot iff a
// uniform word is below the threshold.  q and stack are d-element scratch.
template <typename IdF>
__device__ void vose_build(int32_t d, const double *__restrict__ w, double lam, IdF id, AliasEnt *__restrict__ out,
                           double *__restrict__ q, int32_t *__restrict__ stack) {
    // two stacks in d slots: "small" grows up from the bottom, "large" down from the top
    int32_t ns = 0, nl = 0;
    for (int32_t k = 0; k < d; ++k) {
        const double s = __ddiv_rn(__dmul_rn(w[k], (double)d), lam);
        q[k] = s;
        out[k] = AliasEnt{id(k), 0xFFFFFFFFu};
        if (s < 1.0) stack[ns++] = k;
        else stack[d - 1 - nl++] = k;
    }
    while (ns > 0 && nl > 0) {
        const int32_t sm = stack[--ns];
        const int32_t lg = stack[d - 1 - (--nl)];
        const double qs = q[sm];
        out[sm] = AliasEnt{id(lg), (uint32_t)__double2ull_rz(__dmul_rn(qs, 4294967296.0))};
        const double ql = __dsub_rn(__dadd_rn(q[lg], qs), 1.0);
        q[lg] = ql;
        if (ql < 1.0) stack[ns++] = lg;
        else stack[d - 1 - nl++] = lg;
    }
}

// The same canonical Vose table built by one warp (lane = this thread's lane,
// all 32 lanes call it): the scaled weights, the initial entries and the two
// worklists in index order are written lane-parallel (positions from ballots),
// then lane 0 runs the pairing loop.  Bit-identical to vose_build.
template <typename IdF>
__device__ void vose_build_warp(int32_t d, const double *__restrict__ w, double lam, IdF id, AliasEnt *__restrict__ out,
                                double *__restrict__ q, int32_t *__restrict__ stack, int lane) {
    int32_t ns = 0, nl = 0;  // warp-uniform counts of the small and large lists so far
    const unsigned lt = (1u << lane) - 1u;
    for (int32_t k0 = 0; k0 < d; k0 += 32) {
        const int32_t k = k0 + lane;
        const bool valid = k < d;
        bool small = false;
        if (valid) {
            const double s = __ddiv_rn(__dmul_rn(w[k], (double)d), lam);
            q[k] = s;
            out[k] = AliasEnt{id(k), 0xFFFFFFFFu};
            small = s < 1.0;
        }
        const unsigned sm = __ballot_sync(0xffffffffu, valid && small);
        const unsigned lg = __ballot_sync(0xffffffffu, valid && !small);
        if (valid) {
            if (small) stack[ns + __popc(sm & lt)] = k;
            else stack[d - 1 - (nl + __popc(lg & lt))] = k;
        }
        ns += __popc(sm);
        nl += __popc(lg);
    }
    __syncwarp();
    if (lane == 0) {
        while (ns > 0 && nl > 0) {
            const int32_t s = stack[--ns];
            const int32_t l = stack[d - 1 - (--nl)];
            const double qs = q[s];
            out[s] = AliasEnt{id(l), (uint32_t)__double2ull_rz(__dmul_rn(qs, 4294967296.0))};
            const double ql = __dsub_rn(__dadd_rn(q[l], qs), 1.0);
            q[l] = ql;
            if (ql < 1.0) stack[ns++] = l;
            else stack[d - 1 - nl++] = l;
        }
    }
    __syncwarp();
}

}  // namespace mcx
