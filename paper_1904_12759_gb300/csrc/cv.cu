// Learned control variate (variance reduction, Sec. 5).
//
// Estimator: for any h with h(0) = v, x_i = h(t, i) + E_i[int_0^t W_s R(t - s, X_s) ds]
// with R = A h - dh/dtau (Duhamel's formula with the Feynman-Kac form of
// exp(sA)).  We take h(tau) = v + tau Av + tau^2 A^2v/2 + tau^3 c3 with c3 set so
// that h(t) = xhat, the network's prediction: c3 = (xhat - T2)/t^3,
// T2 = v + t Av + t^2 A^2 v/2, hence R(tau, j) = a_j tau^2 + b_j tau^3 with
// a = A^3 v/2 - 3 c3 and b = A c3.  Over a hold of length D in state j starting
// with remaining time r and log-weight L the residual integral is exactly
//   e^L sum_k c_k D^{k+1} phi_k(delta_j D),   phi_k(z) = int_0^1 e^{zs} s^k ds,
// where R(r - u) = c0 + c1 u + c2 u^2 + c3' u^3.  phi_k: series for |z| <= 1
// (FP32) or 2 (FP64), the recursion phi_k = (e^z - k phi_{k-1})/z otherwise.
//
// Kernels: FP64 SpMV for the Taylor terms; node rates and features
// (double-float sums on the FP32 pipe, FP64 only for rows with values outside
// the double-float range; feature maps in FP32, the network's input
// precision); a 5-64-64-1 ReLU MLP
// (weights rounded to BF16 on load, FP32 accumulation) for prediction,
// full-batch gradients and Adam training (block partial gradients reduced in a
// fixed order: deterministic); the coefficient builder; and the CV walker (the
// FP32 path of the backward walker, with the residual integral in FP32 or FP64).
#include <cuda_bf16.h>
#include <math.h>

#include <algorithm>
#include <new>
#include <type_traits>
#include <vector>

#include "cvmath.cuh"
#include "dfloat.cuh"
#include "expd.cuh"
#include "launch.h"
#include "rows.cuh"
#include "tc.cuh"
#include "walker.cuh"

namespace mcx {
namespace {

constexpr int NF = 5;    // features
constexpr int HID = 64;  // hidden width
constexpr int P_W1 = 0;
constexpr int P_B1 = P_W1 + NF * HID;
constexpr int P_W2 = P_B1 + HID;
constexpr int P_B2 = P_W2 + HID * HID;
constexpr int P_W3 = P_B2 + HID;
constexpr int P_B3 = P_W3 + HID;
constexpr int NPARAM = P_B3 + 1;  // 4609

// ---------------------------------------------------------------------------
// Row passes: Taylor terms, rates, features, cubic coefficients
// ---------------------------------------------------------------------------
// The pre-pass visits each row of A three times: (1) (Av)_i and the rate
// lambda_i; (2) (A^2 v)_i and the features (neighbour statistics of lambda,
// gathered with Av from one 16-byte record per neighbour); (3) (A^3 v)_i (and,
// in the batched form, (A c3)_i from one 16-byte record (A^2 v, c3) per
// neighbour).
//
// Traversal.  Every pass visits the rows in the same way, decided by a row's
// length alone: rows of at most LONG_ROW entries one thread per row, entries
// in order; rows of at most HUGE_ROW entries one warp per row (lanes stride
// the row, xor tree over the lanes); longer rows one block per row (threads
// stride the row; warp trees, then a tree over the warps' results).  A row's
// sums therefore depend only on the row, so two passes (or two layouts) that
// form the same sum get the same bits.  A row schedule lists the rows longer
// than HUGE_ROW, then those longer than LONG_ROW, then the short rows; one
// launch per pass, a static split: blocks take the huge rows, then warps the
// long rows, then groups of 32 short rows.
//
// The short rows are the bulk of a power-law graph and their loads decide the
// time: the matrix entries of 32 rows read one per lane, plus one random
// gather per entry.  Two layouts of the short rows:
//  * CSR (mcx_cv_prepare, mcx_cv_coefficients): short rows in their natural
//    order, so a warp's 32 rows are adjacent in memory;
//  * sliced ELL (the batched form, built once at creation): the same order,
//    stored in chunks of 32 rows with entry k of the chunk's rows contiguous,
//    so that a warp's loads of the matrix are coalesced too.  (Sorting rows by
//    length within windows, so that a warp's lanes run rows of nearly equal
//    length, scatters the per-row reads and writes; measured slower.)
// GB300 runs FP64 at a small fraction of its FP32 rate: the sums' multiply-adds
// stay FP64, but sign tests, the rates and the features run on the integer and
// FP32 pipes (double-float).  A row operation Op supplies
//   Acc zero(); add(acc, i, c, a) per entry (column c, value a);
//   combine(x, y) and shfl(x, o) for the trees; finish(i, acc), one thread.
constexpr int WINDOW = CV_ROW_WINDOW;  // rows per window of the schedule builder (one block per window)
constexpr int PASS_THREADS = 256;
constexpr int PASS_MIN_BLOCKS = 6;

// Row schedule (CvRowSchedule): order [n] = huge rows, long rows, short rows in
// natural order; cnt = {huge, long, short, huge cursor, long cursor}; hist:
// [windows + 1] the windows' starts among the short rows.
using RowSchedule = CvRowSchedule;
static_assert(CV_ROW_CNT >= 5, "row schedule counters");

__device__ __forceinline__ bool is_short(int64_t len) { return len <= LONG_ROW; }

// per window: its number of short rows; global numbers of huge and long rows
__global__ void __launch_bounds__(WINDOW) k_sched_count(int64_t n, const int64_t *__restrict__ rp,
                                                        uint32_t *__restrict__ win, uint32_t *cnt) {
    const int64_t i = (int64_t)blockIdx.x * WINDOW + threadIdx.x;
    int s = 0, l = 0, h = 0;
    if (i < n) {
        const int64_t len = rp[i + 1] - rp[i];
        s = is_short(len);
        h = len > HUGE_ROW;
        l = !s && !h;
    }
    s = __syncthreads_count(s);
    l = __syncthreads_count(l);
    h = __syncthreads_count(h);
    if (threadIdx.x == 0) {
        win[blockIdx.x] = (uint32_t)s;
        if (l) atomicAdd(cnt + 1, (uint32_t)l);
        if (h) atomicAdd(cnt + 0, (uint32_t)h);
    }
}

// exclusive scan of the windows' short counts (one block); cnt[2] = total
__global__ void __launch_bounds__(1024) k_sched_scan(int64_t windows, uint32_t *win, uint32_t *cnt) {
    __shared__ uint32_t part[1024];
    const int64_t per = (windows + 1023) / 1024;
    const int64_t a = (int64_t)threadIdx.x * per, b = a + per < windows ? a + per : windows;
    uint32_t s = 0;
    for (int64_t w = a; w < b; ++w) s += win[w];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {  // inclusive scan of the partial sums
        const uint32_t add = threadIdx.x >= (unsigned)o ? part[threadIdx.x - o] : 0u;
        __syncthreads();
        part[threadIdx.x] += add;
        __syncthreads();
    }
    uint32_t run = threadIdx.x ? part[threadIdx.x - 1] : 0u;
    for (int64_t w = a; w < b; ++w) {
        const uint32_t c = win[w];
        win[w] = run;
        run += c;
    }
    if (threadIdx.x == 1023) cnt[2] = part[1023];
}

// place every row: huge and long rows at their lists' cursors (any order),
// short rows in natural order
__global__ void __launch_bounds__(WINDOW) k_sched_fill(int64_t n, const int64_t *__restrict__ rp,
                                                       const uint32_t *__restrict__ win, uint32_t *cnt,
                                                       int32_t *__restrict__ order) {
    __shared__ uint32_t wc[WINDOW / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t i = (int64_t)blockIdx.x * WINDOW + threadIdx.x;
    const int64_t len = i < n ? rp[i + 1] - rp[i] : -1;
    const bool sh = i < n && is_short(len);
    const unsigned m = __ballot_sync(0xffffffffu, sh);
    if (lane == 0) wc[warp] = (uint32_t)__popc(m);
    __syncthreads();
    uint32_t before = (uint32_t)__popc(m & ((1u << lane) - 1u));
    for (int w = 0; w < warp; ++w) before += wc[w];
    if (i < n) {
        const uint32_t n_huge = cnt[0], n_long = cnt[1];
        if (sh) order[n_huge + n_long + win[blockIdx.x] + before] = (int32_t)i;
        else if (len > HUGE_ROW) order[atomicAdd(cnt + 3, 1u)] = (int32_t)i;
        else order[n_huge + atomicAdd(cnt + 4, 1u)] = (int32_t)i;
    }
}

template <class Op, bool ELL>
__global__ void __launch_bounds__(PASS_THREADS, PASS_MIN_BLOCKS)
    k_pass(const int64_t *__restrict__ rp, const int32_t *__restrict__ col, const double *__restrict__ val,
           const int32_t *__restrict__ order, const uint32_t *__restrict__ cnt, CvSell ell, Op op) {
    __shared__ typename Op::Acc sh[PASS_THREADS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t n_huge = cnt[0], n_long = cnt[1], n_short = cnt[2];
    for (uint32_t r = blockIdx.x; r < n_huge; r += gridDim.x) {
        const int32_t i = order[r];
        typename Op::Acc a = Op::zero();
#pragma unroll 4
        for (int64_t p = rp[i] + threadIdx.x; p < rp[i + 1]; p += PASS_THREADS) op.add(a, i, col[p], val[p]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a = Op::combine(a, Op::shfl(a, o));
        if (lane == 0) sh[warp] = a;
        __syncthreads();
        if (warp == 0) {
            typename Op::Acc s = lane < PASS_THREADS / 32 ? sh[lane] : Op::zero();
#pragma unroll
            for (int o = PASS_THREADS / 64; o > 0; o >>= 1) s = Op::combine(s, Op::shfl(s, o));
            if (lane == 0) op.finish(i, s);
        }
        __syncthreads();  // sh reusable
    }
    const uint32_t warps = gridDim.x * (PASS_THREADS / 32);
    const uint32_t gw = blockIdx.x * (PASS_THREADS / 32) + (uint32_t)warp;
    for (uint32_t k = gw; k < n_long; k += warps) {
        const int32_t i = order[n_huge + k];
        typename Op::Acc a = Op::zero();
#pragma unroll 4
        for (int64_t p = rp[i] + lane; p < rp[i + 1]; p += 32) op.add(a, i, col[p], val[p]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a = Op::combine(a, Op::shfl(a, o));
        if (lane == 0) op.finish(i, a);
    }
    const uint32_t items = (n_short + 31) / 32;
    for (uint32_t k = gw; k < items; k += warps) {
        const uint32_t j = k * 32u + (uint32_t)lane;
        if (j >= n_short) continue;
        const int32_t i = order[n_huge + n_long + j];
        typename Op::Acc a = Op::zero();
        if constexpr (ELL) {
            const int d = ell.len[j];
            const int32_t *c = ell.col + ell.chunk[k] + lane;
            const double *w = ell.val + ell.chunk[k] + lane;
            // two entries per iteration (measured on BA n = 4e6: unroll 1 / 2 / 4 / 8 gave
            // 1.92 / 1.77 / 1.84 / 1.93 ms per learned-CV run)
#pragma unroll 2
            for (int e = 0; e < d; ++e) op.add(a, i, c[32 * e], w[32 * e]);
        } else {
            const int64_t p0 = rp[i], p1 = rp[i + 1];
#pragma unroll 4
            for (int64_t p = p0; p < p1; ++p) op.add(a, i, col[p], val[p]);
        }
        op.finish(i, a);
    }
}

unsigned pass_grid() { return 152u * PASS_MIN_BLOCKS; }

// Build the row schedule of rows 0..n-1 (short rows in natural order).
cudaError_t build_schedule(int64_t n, const int64_t *rp, const RowSchedule &s, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(s.cnt, 0, sizeof(uint32_t) * CV_ROW_CNT, st);
    if (e != cudaSuccess) return e;
    const int64_t windows = (n + WINDOW - 1) / WINDOW;
    k_sched_count<<<(unsigned)windows, WINDOW, 0, st>>>(n, rp, s.hist, s.cnt);
    k_sched_scan<<<1, 1024, 0, st>>>(windows, s.hist, s.cnt);
    k_sched_fill<<<(unsigned)windows, WINDOW, 0, st>>>(n, rp, s.hist, s.cnt, s.order);
    return cudaGetLastError();
}

// One pass of `op` over the scheduled rows; ell: the short rows' sliced ELL
// copy, or NULL (CSR).
template <class Op>
void run_pass(const int64_t *rp, const int32_t *col, const double *val, const RowSchedule &s, const CvSell *ell,
              const Op &op, cudaStream_t st) {
    if (ell)
        k_pass<Op, true><<<pass_grid(), PASS_THREADS, 0, st>>>(rp, col, val, s.order, s.cnt, *ell, op);
    else
        k_pass<Op, false><<<pass_grid(), PASS_THREADS, 0, st>>>(rp, col, val, s.order, s.cnt, CvSell{}, op);
}

// a > 0 for a double by its bits (integer pipe): sign clear, not zero, not NaN
__device__ __forceinline__ bool positive(double a) {
    const long long b = __double_as_longlong(a);
    return b > 0 && b <= 0x7ff0000000000000ll;
}

__device__ __forceinline__ df df_shfl(df a, int o) { return df_shfl_xor(a, o); }

// A double-float value in the second half of a 16-byte record (h in the low word).
__device__ __forceinline__ double df_pack(df a) { return __hiloint2double(__float_as_int(a.l), __float_as_int(a.h)); }
__device__ __forceinline__ df df_unpack(double d) {
    return df{__int_as_float(__double2loint(d)), __int_as_float(__double2hiint(d))};
}

// rate lambda_i = sum of the positive off-diagonal entries in FP64, entry order
// (rows with a value outside the double-float range)
__device__ __forceinline__ double rate_fp64(int64_t i, const int64_t *__restrict__ rp,
                                            const int32_t *__restrict__ col, const double *__restrict__ val) {
    double s = 0.0;
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p)
        if (col[p] != i && positive(val[p])) s = __dadd_rn(s, val[p]);
    return s;
}

// Pass 1 on row i: (Av)_i (FP64) and lambda_i (double-float sum of the kept
// entries, FP64 where a value is outside the double-float range).  Writes Av,
// lambda (FP64) and the record g_i = (Av_i, lambda_i as double-float) for pass
// 2, whose high part is a NaN where lambda_i is outside 2^-60 .. 2^60 (pass 2
// squares it), so that pass 2 takes that row's neighbours in FP64.
struct PassRates {
    const int64_t *rp;
    const int32_t *col;
    const double *val;
    const double *x;  // v
    double *t1;       // Av
    double *lam;      // lambda (FP64)
    double2 *g;       // (Av_i, lambda_i)
    struct Acc {
        double t;
        df s;
        int bad;
    };
    static __device__ __forceinline__ Acc zero() { return Acc{0.0, {0.0f, 0.0f}, 0}; }
    __device__ __forceinline__ void add(Acc &a, int64_t i, int32_t c, double w) const {
        a.t = __fma_rn(w, __ldg(x + c), a.t);
        if (c != i && positive(w)) {
            bool b = false;
            a.s = df_add(a.s, df_split(w, b));
            a.bad |= (int)b;
        }
    }
    static __device__ __forceinline__ Acc shfl(Acc a, int o) {
        return Acc{__shfl_xor_sync(0xffffffffu, a.t, o), df_shfl(a.s, o), __shfl_xor_sync(0xffffffffu, a.bad, o)};
    }
    static __device__ __forceinline__ Acc combine(Acc a, Acc b) { return Acc{a.t + b.t, df_add(a.s, b.s), a.bad | b.bad}; }
    __device__ __forceinline__ void finish(int64_t i, Acc a) const {
        df d;
        double l;
        bool b = false;
        if (a.bad) {
            l = rate_fp64(i, rp, col, val);
            d = df_split(l, b);
        } else {
            d = df_norm(a.s);
            l = df_to_double(d);
        }
        const float m = fabsf(d.h);
        if (b || !(m == 0.0f || (m >= 8.673617379884035e-19f && m <= 1.152921504606847e18f)))
            d.h = __int_as_float(0x7fc00000);
        t1[i] = a.t;
        lam[i] = l;
        g[i] = make_double2(a.t, df_pack(d));
    }
};

// Features of node i, mapped to FP32: log1p(lambda), log1p(mean and standard
// deviation of the neighbours' lambda), t Av / T2, t^2 A^2 v / (2 T2) with
// T2 = v + t Av + t^2 A^2 v/2.  T2 and the two numerators in double-float on
// the FP32 pipe where every input and intermediate stays well inside its
// range (2^-90 .. 2^100), else in FP64.
__device__ __forceinline__ bool df_safe(df a) {
    const float m = fabsf(a.h);
    return m == 0.0f || (m >= 8.077935669463161e-28f && m <= 1.2676506002282294e30f);
}

__device__ __forceinline__ void feature_row(int64_t i, float mean, float sd, float lam_i, double v_i, double t1,
                                            double t2, double t, float *__restrict__ F) {
    bool bad = false;
    const df dv = df_split(v_i, bad), d1 = df_split(t1, bad), d2 = df_split(t2, bad), dt = df_split(t, bad);
    const df a1 = df_mul(dt, d1);              // t Av
    const df a2 = df_mul(df_mul(dt, dt), d2);  // t^2 A^2 v
    const df T2 = df_norm(df_add(df_add(dv, a1), df{__fmul_rn(0.5f, a2.h), __fmul_rn(0.5f, a2.l)}));
    float n3, n4, T2s;
    if (!bad && df_safe(dv) && df_safe(a1) && df_safe(a2) && df_safe(T2)) {
        n3 = __fadd_rn(a1.h, a1.l);
        n4 = __fadd_rn(a2.h, a2.l);
        T2s = T2.h != 0.0f ? T2.h : 1.0f;
    } else {
        const double T2d = v_i + t * t1 + t * t * t2 / 2.0;
        n3 = (float)(t * t1);
        n4 = (float)(t * t * t2);
        T2s = T2d != 0.0 ? (float)T2d : 1.0f;
    }
    float *f = F + i * NF;
    f[0] = log1pf(lam_i);
    f[1] = log1pf(mean);
    f[2] = log1pf(sd);
    f[3] = __fdiv_rn(n3, T2s);
    f[4] = __fdiv_rn(n4, __fmul_rn(2.0f, T2s));
}

// Pass 2 on row i: (A^2 v)_i (FP64) and the features.  The neighbours' lambda
// sums s1 = sum lambda_c, s2 = sum lambda_c^2 over the kept entries in
// double-float; where either is not finite (a neighbour's lambda outside the
// double-float range, or an overflow) the row's statistics are redone in FP64.
struct PassFeatures {
    const int64_t *rp;
    const int32_t *col;
    const double *val;
    const double2 *g;   // pass 1's records
    const double *v;
    const double *lam;  // FP64 lambda
    double *t2;         // A^2 v
    float *F;
    double t_all;
    const double *t_row;  // per-row horizon, or NULL (t_all)
    struct Acc {
        double t;
        df s1, s2;
        int d;
    };
    static __device__ __forceinline__ Acc zero() { return Acc{0.0, {0.0f, 0.0f}, {0.0f, 0.0f}, 0}; }
    __device__ __forceinline__ void add(Acc &a, int64_t i, int32_t c, double w) const {
        const double2 q = __ldg(g + c);
        a.t = __fma_rn(w, q.x, a.t);
        if (c != i && positive(w)) {
            const df x = df_unpack(q.y);
            a.s1 = df_add(a.s1, x);
            a.s2 = df_add(a.s2, df_mul(x, x));
            a.d += 1;
        }
    }
    static __device__ __forceinline__ Acc shfl(Acc a, int o) {
        return Acc{__shfl_xor_sync(0xffffffffu, a.t, o), df_shfl(a.s1, o), df_shfl(a.s2, o),
                   __shfl_xor_sync(0xffffffffu, a.d, o)};
    }
    static __device__ __forceinline__ Acc combine(Acc a, Acc b) {
        return Acc{a.t + b.t, df_add(a.s1, b.s1), df_add(a.s2, b.s2), a.d + b.d};
    }
    __device__ __forceinline__ void finish(int64_t i, Acc a) const {
        float mean = 0.0f, sd = 0.0f;
        const bool bad = !(fabsf(a.s1.h) <= 3.4028234663852886e38f) || !(fabsf(a.s2.h) <= 3.4028234663852886e38f);
        if (bad) {
            double s1 = 0.0, s2 = 0.0, d = 0.0;
            for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
                const int32_t c = col[p];
                if (c != i && positive(val[p])) {
                    s1 += lam[c];
                    s2 += lam[c] * lam[c];
                    d += 1.0;
                }
            }
            const double m = d > 0.0 ? s1 / d : 0.0;
            const double var = d > 0.0 ? s2 / d - m * m : 0.0;
            mean = (float)m;
            sd = var > 0.0 ? (float)sqrt(var) : 0.0f;
        } else if (a.d > 0) {
            const float d = (float)a.d;  // exact: rows have fewer than 2^24 entries
            // mean = s1/d and var = s2/d - mean^2 in double-float (one correction step per quotient)
            const float m1 = __fdiv_rn(a.s1.h, d);
            const df mu = df{m1, __fdiv_rn(__fadd_rn(__fmaf_rn(-m1, d, a.s1.h), a.s1.l), d)};
            const float m2 = __fdiv_rn(a.s2.h, d);
            const df q2 = df{m2, __fdiv_rn(__fadd_rn(__fmaf_rn(-m2, d, a.s2.h), a.s2.l), d)};
            const df mm = df_mul(mu, mu);
            const df var = df_norm(df_add(q2, df{-mm.h, -mm.l}));
            mean = __fadd_rn(mu.h, mu.l);
            sd = var.h > 0.0f ? sqrtf(var.h) : 0.0f;
        }
        t2[i] = a.t;
        const double2 gi = g[i];
        const df li = df_unpack(gi.y);
        const float lf = li.h == li.h ? __fadd_rn(li.h, li.l) : (float)lam[i];
        feature_row(i, mean, sd, lf, v[i], gi.x, a.t, t_row ? t_row[i] : t_all, F);
    }
};

// y = A x as a row pass.
struct PassSpmv {
    const double *x;
    double *y;
    struct Acc {
        double t;
    };
    static __device__ __forceinline__ Acc zero() { return Acc{0.0}; }
    __device__ __forceinline__ void add(Acc &a, int64_t, int32_t c, double w) const {
        a.t = __fma_rn(w, __ldg(x + c), a.t);
    }
    static __device__ __forceinline__ Acc shfl(Acc a, int o) { return Acc{__shfl_xor_sync(0xffffffffu, a.t, o)}; }
    static __device__ __forceinline__ Acc combine(Acc a, Acc b) { return Acc{a.t + b.t}; }
    __device__ __forceinline__ void finish(int64_t i, Acc a) const { y[i] = a.t; }
};

// Pass 3 of the batched form on row i: (A^3 v)_i and (A c3)_i from the records
// q_c = (A^2 v_c, c3_c), each sum formed as PassSpmv forms it, then the
// coefficient pair (a_i, b_i) = (A^3 v_i / 2 - 3 c3_i, (A c3)_i), as k_cv_ab
// forms it from those sums.
struct PassCubic {
    const double2 *q;
    double2 *ab;
    struct Acc {
        double t, b;
    };
    static __device__ __forceinline__ Acc zero() { return Acc{0.0, 0.0}; }
    __device__ __forceinline__ void add(Acc &a, int64_t, int32_t c, double w) const {
        const double2 r = __ldg(q + c);
        a.t = __fma_rn(w, r.x, a.t);
        a.b = __fma_rn(w, r.y, a.b);
    }
    static __device__ __forceinline__ Acc shfl(Acc a, int o) {
        return Acc{__shfl_xor_sync(0xffffffffu, a.t, o), __shfl_xor_sync(0xffffffffu, a.b, o)};
    }
    static __device__ __forceinline__ Acc combine(Acc a, Acc b) { return Acc{a.t + b.t, a.b + b.b}; }
    __device__ __forceinline__ void finish(int64_t i, Acc a) const {
        ab[i] = make_double2(a.t / 2.0 - 3.0 * q[i].y, a.b);
    }
};

// ---------------------------------------------------------------------------
// MLP
// ---------------------------------------------------------------------------
__device__ __forceinline__ float bf16_round(float x) {
    uint32_t u = __float_as_uint(x);
    u = (u + 0x7FFFu + ((u >> 16) & 1u)) & 0xFFFF0000u;
    return __uint_as_float(u);
}

struct MLPView {
    const float *params;  // FP32 master (weights rounded to BF16 when loaded)
    const float *mu;      // [NF] feature means
    const float *sd;      // [NF] feature standard deviations
};

// x = (f - mu) * (1/sd), isd = 1/sd rounded to FP32 (the same in training and inference)
__device__ __forceinline__ void standardise(const float *__restrict__ f, const float *mu, const float *isd,
                                           float x[NF]) {
#pragma unroll
    for (int q = 0; q < NF; ++q) x[q] = __fmul_rn(__fsub_rn(f[q], mu[q]), isd[q]);
}

// ---------------------------------------------------------------------------
// Inference on the tensor cores.  A CTA of 4 warps takes tiles of 128 nodes:
// each thread computes its node's first hidden layer (5 -> 64, FP32 CUDA
// cores, BF16 weights) and writes it, rounded to BF16, as row `tid` of the MMA
// operand A (128 x 64, K-major core-matrix layout in shared memory); one
// thread issues four 128 x 64 x 16 BF16 MMAs against W2 (resident in shared
// memory as the K-major operand B = W2^T) into 64 TMEM columns of FP32
// accumulators, committed to an mbarrier; each warp then reads its 32 TMEM
// lanes (= its 32 nodes) and finishes bias, ReLU and the 64 -> 1 output layer.
// ---------------------------------------------------------------------------
constexpr int TC_ROWS = 128;        // nodes per tile (MMA M)
constexpr uint32_t TC_COLS = 64;    // TMEM columns (MMA N, FP32 accumulators)
constexpr uint32_t TC_WAIT = 1u << 22;  // mbarrier polls before giving up

// byte offset of element (r, k) in a K-major no-swizzle operand with 64 K
// elements per row: 8-row groups 1024 B apart, K-adjacent core matrices 128 B apart
__device__ __forceinline__ uint32_t tc_off(uint32_t r, uint32_t k) {
    return (r >> 3) * 1024u + (k >> 3) * 128u + (r & 7u) * 16u + (k & 7u) * 2u;
}

__device__ __forceinline__ uint32_t bf16_bits(float x) {
    const uint32_t u = __float_as_uint(x);
    return (u + 0x7FFFu + ((u >> 16) & 1u)) >> 16;
}

__global__ void __launch_bounds__(TC_ROWS, 7) k_mlp_predict_tc(int64_t n, const float *__restrict__ F, MLPView m,
                                                               float *__restrict__ y, uint32_t *err,
                                                               uint32_t wait_polls) {
    __shared__ __align__(1024) uint8_t sA[TC_ROWS * HID * 2];  // 16 KB
    __shared__ __align__(1024) uint8_t sB[HID * HID * 2];      // 8 KB
    __shared__ __align__(16) float sW1[NF * HID];
    __shared__ __align__(16) float sb1[HID];
    __shared__ __align__(16) float sb2[HID];
    __shared__ __align__(16) float sw3[HID];
    __shared__ float sb3, smu[NF], sisd[NF];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5;
    for (int k = tid; k < HID * HID; k += TC_ROWS) {  // B[n][j] = W2[j][n]
        const int j = k / HID, nn = k % HID;
        *reinterpret_cast<uint16_t *>(sB + tc_off(nn, j)) = (uint16_t)bf16_bits(m.params[P_W2 + k]);
    }
    for (int k = tid; k < NF * HID; k += TC_ROWS) sW1[k] = bf16_round(m.params[P_W1 + k]);
    if (tid < HID) {
        sb1[tid] = m.params[P_B1 + tid];
        sb2[tid] = m.params[P_B2 + tid];
        sw3[tid] = bf16_round(m.params[P_W3 + tid]);
    }
    if (tid < NF) {
        smu[tid] = m.mu[tid];
        sisd[tid] = __fdiv_rn(1.0f, m.sd[tid]);
    }
    if (tid == 0) {
        sb3 = m.params[P_B3];
        tc::mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tc::tmem_alloc(&tmem_base, TC_COLS);
    tc::fence_proxy_async_smem();  // B written by this thread's generic stores
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_base;
    const uint32_t a_addr = tc::smem_addr(sA), b_addr = tc::smem_addr(sB);
    constexpr uint32_t idesc = tc::idesc_bf16_f32(TC_ROWS, TC_COLS);
    uint32_t phase = 0;
    for (int64_t tile = blockIdx.x; tile * TC_ROWS < n; tile += gridDim.x) {
        const int64_t i = tile * TC_ROWS + tid;
        float x[NF] = {0.f, 0.f, 0.f, 0.f, 0.f};
        if (i < n) standardise(F + i * NF, smu, sisd, x);
        // first hidden layer, BF16 (round to nearest even), 16 bytes (8 K elements) per
        // store; the weights and biases read as 16-byte vectors
#pragma unroll
        for (int kc = 0; kc < HID; kc += 8) {
            float a[8];
            *reinterpret_cast<float4 *>(a) = *reinterpret_cast<const float4 *>(sb1 + kc);
            *reinterpret_cast<float4 *>(a + 4) = *reinterpret_cast<const float4 *>(sb1 + kc + 4);
#pragma unroll
            for (int f = 0; f < NF; ++f) {
                const float4 w0 = *reinterpret_cast<const float4 *>(sW1 + f * HID + kc);
                const float4 w1 = *reinterpret_cast<const float4 *>(sW1 + f * HID + kc + 4);
                a[0] = fmaf(x[f], w0.x, a[0]);
                a[1] = fmaf(x[f], w0.y, a[1]);
                a[2] = fmaf(x[f], w0.z, a[2]);
                a[3] = fmaf(x[f], w0.w, a[3]);
                a[4] = fmaf(x[f], w1.x, a[4]);
                a[5] = fmaf(x[f], w1.y, a[5]);
                a[6] = fmaf(x[f], w1.z, a[6]);
                a[7] = fmaf(x[f], w1.w, a[7]);
            }
            uint32_t pk[4];
#pragma unroll
            for (int q = 0; q < 8; q += 2) {
                const __nv_bfloat162 h2 = __floats2bfloat162_rn(fmaxf(a[q], 0.0f), fmaxf(a[q + 1], 0.0f));
                pk[q >> 1] = *reinterpret_cast<const uint32_t *>(&h2);
            }
            *reinterpret_cast<uint4 *>(sA + tc_off((uint32_t)tid, (uint32_t)kc)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
        }
        tc::fence_proxy_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after_sync();
#pragma unroll
            for (uint32_t kk = 0; kk < HID / 16; ++kk)
                tc::mma_bf16(tmem, tc::smem_desc(a_addr + kk * 256u, 128u, 1024u),
                             tc::smem_desc(b_addr + kk * 256u, 128u, 1024u), idesc, kk > 0);
            tc::mma_commit(&bar);
        }
        const bool got = tc::mbar_wait(&bar, phase, wait_polls);
        if (__syncthreads_or(!got)) {
            // the MMAs did not complete within the limit: flag, wait (bounded) for the MMAs
            // in flight to land before the tensor memory is freed, stop
            if (tid == 0) atomicOr(err, 1u);
            tc::mbar_wait(&bar, phase, TC_WAIT);
            break;
        }
        phase ^= 1u;
        tc::fence_after_sync();
        float yv = sb3;
#pragma unroll
        for (uint32_t c = 0; c < TC_COLS; c += 16) {
            float v[16];
            tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + c, v);
            tc::tmem_ld_wait();
            float b2[16], w3[16];
#pragma unroll
            for (int k = 0; k < 16; k += 4) {
                *reinterpret_cast<float4 *>(b2 + k) = *reinterpret_cast<const float4 *>(sb2 + c + k);
                *reinterpret_cast<float4 *>(w3 + k) = *reinterpret_cast<const float4 *>(sw3 + c + k);
            }
#pragma unroll
            for (int k = 0; k < 16; ++k) yv = fmaf(fmaxf(v[k] + b2[k], 0.0f), w3[k], yv);
        }
        if (i < n) y[i] = yv;
        tc::fence_before_sync();
        __syncthreads();  // TMEM read and A consumed before the next tile overwrites them
    }
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tmem, TC_COLS);
}

// ---------------------------------------------------------------------------
// Gradient on the tensor cores.  A CTA of 4 warps takes a tile of 128 samples,
// one per thread, and writes its partial gradient (and loss) to part[tile]:
//  * forward as in inference: the first layer on CUDA cores (FP32, BF16
//    weights), h1 rounded to BF16 into A1 = [samples x 64] and into the
//    transposed operand H1T = [units x samples]; MMA z2 = h1 W2 (128 x 64 x 64,
//    TMEM columns 0..63); bias, ReLU and the output layer on CUDA cores;
//  * backward: dy = 2 (y - target) / batch, dh2 = dy w3 [z2 > 0] rounded to
//    BF16 into D2 = [samples x 64] and D2T = [units x samples]; two MMAs:
//    dh1 = dh2 W2^T (128 x 64 x 64, columns 64..127) and
//    [dW2 ; db2] = [h1^T ; 1] dh2 (128 x 64 x 128 over the tile's samples: rows
//    0..63 of H1T are h1^T, row 64 ones, the rest zero; columns 128..191);
//  * dW1, db1 (from dh1 masked by z1 > 0), dW3, db3 and the loss on CUDA cores
//    in FP32 over the tile (shared memory, fixed order).
// All operands K-major without swizzle; K = 64 operands have their 8-row groups
// 1024 bytes apart, K = 128 operands (samples as K) 2048 bytes apart.
// ---------------------------------------------------------------------------
constexpr int TG_ROWS = 128;  // samples per tile (MMA M)
constexpr uint32_t TG_COLS = 256;  // TMEM columns allocated (three 64-column accumulators)
constexpr int TG_FS = HID + 1;     // row stride of the FP32 per-sample arrays

// byte offset of element (r, k) in a K-major no-swizzle operand with 128 K
// elements per row: 8-row groups 2048 B apart, K-adjacent core matrices 128 B apart
__device__ __forceinline__ uint32_t tc_off128(uint32_t r, uint32_t k) {
    return (r >> 3) * 2048u + (k >> 3) * 128u + (r & 7u) * 16u + (k & 7u) * 2u;
}

// dynamic shared memory of k_mlp_grad_tc (byte offsets; operands 1024-aligned)
constexpr uint32_t TG_W2T = 0;                            // [64 x 64] bf16, (k, j) = W2[j][k]
constexpr uint32_t TG_W2 = TG_W2T + 64 * 64 * 2;          // [64 x 64] bf16, (j, k) = W2[j][k]
constexpr uint32_t TG_A1 = TG_W2 + 64 * 64 * 2;           // [128 x 64] bf16, (s, j) = h1[s][j]
constexpr uint32_t TG_D2 = TG_A1 + 128 * 64 * 2;          // [128 x 64] bf16, (s, k) = dh2[s][k]
constexpr uint32_t TG_H1T = TG_D2 + 128 * 64 * 2;         // [128 x 128] bf16, (j, s) = h1[s][j]; row 64 ones
constexpr uint32_t TG_D2T = TG_H1T + 128 * 128 * 2;       // [64 x 128] bf16, (k, s) = dh2[s][k]
constexpr uint32_t TG_F = TG_D2T + 64 * 128 * 2;          // [128][65] f32: h2, then dh1
constexpr uint32_t TG_X = TG_F + TG_ROWS * TG_FS * 4;     // [128][5] f32 standardised inputs
constexpr uint32_t TG_DY = TG_X + TG_ROWS * NF * 4;       // [128] f32 dy
constexpr uint32_t TG_LS = TG_DY + TG_ROWS * 4;           // [128] f32 squared residuals
constexpr uint32_t TG_W1 = TG_LS + TG_ROWS * 4;           // [5 x 64] f32 (BF16-rounded)
constexpr uint32_t TG_B1 = TG_W1 + NF * HID * 4;          // [64] f32
constexpr uint32_t TG_B2 = TG_B1 + HID * 4;               // [64] f32
constexpr uint32_t TG_W3 = TG_B2 + HID * 4;               // [64] f32 (BF16-rounded)
constexpr uint32_t TG_SMEM = TG_W3 + HID * 4;

__global__ void __launch_bounds__(TG_ROWS, 1) k_mlp_grad_tc(int64_t n, const float *__restrict__ F,
                                                          const float *__restrict__ tgt,
                                                          const int64_t *__restrict__ idx, MLPView m,
                                                          float inv_batch, float *__restrict__ part, uint32_t *err,
                                                          uint32_t wait_polls) {
    extern __shared__ __align__(1024) uint8_t sm[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tmem_base;
    __shared__ float sb3, smu[NF], sisd[NF];
    float *sF = reinterpret_cast<float *>(sm + TG_F);
    float *sX = reinterpret_cast<float *>(sm + TG_X);
    float *sDY = reinterpret_cast<float *>(sm + TG_DY);
    float *sLS = reinterpret_cast<float *>(sm + TG_LS);
    float *sW1 = reinterpret_cast<float *>(sm + TG_W1);
    float *sb1 = reinterpret_cast<float *>(sm + TG_B1);
    float *sb2 = reinterpret_cast<float *>(sm + TG_B2);
    float *sw3 = reinterpret_cast<float *>(sm + TG_W3);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // ---- weights (BF16 as used), the constant rows of H1T, TMEM, mbarrier ----
    for (int k = tid; k < HID * HID; k += TG_ROWS) {
        const int j = k / HID, kk = k % HID;
        const uint16_t w = (uint16_t)bf16_bits(m.params[P_W2 + k]);  // W2[j][kk]
        *reinterpret_cast<uint16_t *>(sm + TG_W2T + tc_off((uint32_t)kk, (uint32_t)j)) = w;
        *reinterpret_cast<uint16_t *>(sm + TG_W2 + tc_off((uint32_t)j, (uint32_t)kk)) = w;
    }
    for (int k = tid; k < NF * HID; k += TG_ROWS) sW1[k] = bf16_round(m.params[P_W1 + k]);
    if (tid < HID) {
        sb1[tid] = m.params[P_B1 + tid];
        sb2[tid] = m.params[P_B2 + tid];
        sw3[tid] = bf16_round(m.params[P_W3 + tid]);
    }
    for (int r = HID; r < TG_ROWS; ++r)  // row 64 of H1T: ones (db2); rows 65..127: zero
        *reinterpret_cast<uint16_t *>(sm + TG_H1T + tc_off128((uint32_t)r, (uint32_t)tid)) =
            r == HID ? (uint16_t)0x3F80u : (uint16_t)0u;
    if (tid < NF) {
        smu[tid] = m.mu[tid];
        sisd[tid] = __fdiv_rn(1.0f, m.sd[tid]);
    }
    if (tid == 0) {
        sb3 = m.params[P_B3];
        tc::mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tc::tmem_alloc(&tmem_base, TG_COLS);
    __syncthreads();
    // ---- forward: first layer (FP32, BF16 weights), h1 to both operands ----
    const int64_t smp = (int64_t)blockIdx.x * TG_ROWS + tid;
    const bool valid = smp < n;
    float x[NF] = {0.f, 0.f, 0.f, 0.f, 0.f};
    float target = 0.0f;
    if (valid) {
        const int64_t row = idx ? idx[smp] : smp;
        standardise(F + row * NF, smu, sisd, x);
        target = tgt[row];
    }
#pragma unroll
    for (int f = 0; f < NF; ++f) sX[tid * NF + f] = x[f];
    uint32_t mask1[2] = {0u, 0u};  // z1 > 0, bit per hidden unit
#pragma unroll
    for (int kc = 0; kc < HID; kc += 8) {
        float a[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) a[q] = sb1[kc + q];
#pragma unroll
        for (int f = 0; f < NF; ++f)
#pragma unroll
            for (int q = 0; q < 8; ++q) a[q] = fmaf(x[f], sW1[f * HID + kc + q], a[q]);
        uint32_t pk[4];
#pragma unroll
        for (int q = 0; q < 8; q += 2) {
            const __nv_bfloat162 h2v = __floats2bfloat162_rn(fmaxf(a[q], 0.0f), fmaxf(a[q + 1], 0.0f));
            pk[q >> 1] = *reinterpret_cast<const uint32_t *>(&h2v);
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            if (a[q] > 0.0f) mask1[(kc + q) >> 5] |= 1u << ((kc + q) & 31);
            const uint16_t hb = (uint16_t)(pk[q >> 1] >> ((q & 1) * 16));
            *reinterpret_cast<uint16_t *>(sm + TG_H1T + tc_off128((uint32_t)(kc + q), (uint32_t)tid)) = hb;
        }
        *reinterpret_cast<uint4 *>(sm + TG_A1 + tc_off((uint32_t)tid, (uint32_t)kc)) =
            make_uint4(pk[0], pk[1], pk[2], pk[3]);
    }
    tc::fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_base;
    constexpr uint32_t idesc = tc::idesc_bf16_f32(TG_ROWS, 64);
    const uint32_t base = tc::smem_addr(sm);
    if (tid == 0) {  // z2 = h1 W2
#pragma unroll
        for (uint32_t kk = 0; kk < HID / 16; ++kk)
            tc::mma_bf16(tmem, tc::smem_desc(base + TG_A1 + kk * 256u, 128u, 1024u),
                         tc::smem_desc(base + TG_W2T + kk * 256u, 128u, 1024u), idesc, kk > 0);
        tc::mma_commit(&bar);
    }
    bool ok = tc::mbar_wait(&bar, 0u, wait_polls);
    if (__syncthreads_or(!ok)) {
        if (tid == 0) atomicOr(err, 2u);
        tc::mbar_wait(&bar, 0u, TC_WAIT);
    } else {
        tc::fence_after_sync();
        // ---- output layer and the backward signal dh2 ----
        const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
        float z[HID];
#pragma unroll
        for (uint32_t c = 0; c < HID; c += 16) tc::tmem_ld16(tmem + lane_base + c, z + c);
        tc::tmem_ld_wait();
        float y = sb3;
#pragma unroll
        for (int k = 0; k < HID; ++k) {
            z[k] = z[k] + sb2[k];
            const float h = fmaxf(z[k], 0.0f);
            sF[tid * TG_FS + k] = h;
            y = fmaf(h, sw3[k], y);
        }
        const float r = valid ? y - target : 0.0f;
        const float dy = 2.0f * r * inv_batch;
        sDY[tid] = dy;
        sLS[tid] = r * r;
#pragma unroll
        for (int kc = 0; kc < HID; kc += 8) {
            uint32_t pk[4];
#pragma unroll
            for (int q = 0; q < 8; q += 2) {
                const float d0 = z[kc + q] > 0.0f ? dy * sw3[kc + q] : 0.0f;
                const float d1 = z[kc + q + 1] > 0.0f ? dy * sw3[kc + q + 1] : 0.0f;
                const __nv_bfloat162 dv = __floats2bfloat162_rn(d0, d1);
                pk[q >> 1] = *reinterpret_cast<const uint32_t *>(&dv);
            }
#pragma unroll
            for (int q = 0; q < 8; ++q)
                *reinterpret_cast<uint16_t *>(sm + TG_D2T + tc_off128((uint32_t)(kc + q), (uint32_t)tid)) =
                    (uint16_t)(pk[q >> 1] >> ((q & 1) * 16));
            *reinterpret_cast<uint4 *>(sm + TG_D2 + tc_off((uint32_t)tid, (uint32_t)kc)) =
                make_uint4(pk[0], pk[1], pk[2], pk[3]);
        }
        tc::fence_proxy_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (tid == 0) {  // dh1 = dh2 W2^T;  [dW2 ; db2] = [h1^T ; 1] dh2 over the tile's samples
#pragma unroll
            for (uint32_t kk = 0; kk < HID / 16; ++kk)
                tc::mma_bf16(tmem + 64u, tc::smem_desc(base + TG_D2 + kk * 256u, 128u, 1024u),
                             tc::smem_desc(base + TG_W2 + kk * 256u, 128u, 1024u), idesc, kk > 0);
#pragma unroll
            for (uint32_t kk = 0; kk < TG_ROWS / 16; ++kk)
                tc::mma_bf16(tmem + 128u, tc::smem_desc(base + TG_H1T + kk * 256u, 128u, 2048u),
                             tc::smem_desc(base + TG_D2T + kk * 256u, 128u, 2048u), idesc, kk > 0);
            tc::mma_commit(&bar);
        }
        // meanwhile: dW3, db3 and the loss over the tile (FP32, sample order)
        float *out = part + (int64_t)blockIdx.x * (NPARAM + 1);
        if (tid < HID) {
            float g = 0.0f;
            for (int s = 0; s < TG_ROWS; ++s) g = fmaf(sF[s * TG_FS + tid], sDY[s], g);
            out[P_W3 + tid] = g;
        } else if (tid == HID) {
            float gb3 = 0.0f, loss = 0.0f;
            for (int s = 0; s < TG_ROWS; ++s) {
                gb3 += sDY[s];
                loss += sLS[s];
            }
            out[P_B3] = gb3;
            out[NPARAM] = loss * inv_batch;
        }
        ok = tc::mbar_wait(&bar, 1u, wait_polls);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) atomicOr(err, 2u);
            tc::mbar_wait(&bar, 1u, TC_WAIT);
        } else {
            tc::fence_after_sync();
            // dh1 (masked by z1 > 0) to shared memory for dW1 and db1
#pragma unroll
            for (uint32_t c = 0; c < HID; c += 16) {
                float v[16];
                tc::tmem_ld16(tmem + lane_base + 64u + c, v);
                tc::tmem_ld_wait();
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    const int j = (int)c + k;
                    sF[tid * TG_FS + j] = ((mask1[j >> 5] >> (j & 31)) & 1u) ? v[k] : 0.0f;
                }
            }
            // dW2 (TMEM rows 0..63) and db2 (row 64), one row per thread of warps 0..2
#pragma unroll
            for (uint32_t c = 0; c < HID; c += 16) {
                float v[16];
                tc::tmem_ld16(tmem + lane_base + 128u + c, v);
                tc::tmem_ld_wait();
                const int row = warp * 32 + lane;
                if (row < HID) {
#pragma unroll
                    for (int k = 0; k < 16; ++k) out[P_W2 + row * HID + (int)c + k] = v[k];
                } else if (row == HID) {
#pragma unroll
                    for (int k = 0; k < 16; ++k) out[P_B2 + (int)c + k] = v[k];
                }
            }
            __syncthreads();
            {  // dW1 and db1: thread t sums column j = t mod 64 over the tile, half the outputs each
                const int j = tid & (HID - 1);
                if (tid < HID) {
                    float g0 = 0.0f, g1 = 0.0f, g2 = 0.0f;
                    for (int s = 0; s < TG_ROWS; ++s) {
                        const float d = sF[s * TG_FS + j];
                        g0 = fmaf(sX[s * NF + 0], d, g0);
                        g1 = fmaf(sX[s * NF + 1], d, g1);
                        g2 = fmaf(sX[s * NF + 2], d, g2);
                    }
                    out[P_W1 + 0 * HID + j] = g0;
                    out[P_W1 + 1 * HID + j] = g1;
                    out[P_W1 + 2 * HID + j] = g2;
                } else {
                    float g3 = 0.0f, g4 = 0.0f, gb = 0.0f;
                    for (int s = 0; s < TG_ROWS; ++s) {
                        const float d = sF[s * TG_FS + j];
                        g3 = fmaf(sX[s * NF + 3], d, g3);
                        g4 = fmaf(sX[s * NF + 4], d, g4);
                        gb += d;
                    }
                    out[P_W1 + 3 * HID + j] = g3;
                    out[P_W1 + 4 * HID + j] = g4;
                    out[P_B1 + j] = gb;
                }
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tmem, TG_COLS);
}

// Sum the block partials in block order (deterministic); optionally apply Adam.
__global__ void k_grad_reduce(int nblocks, const float *__restrict__ part, float *__restrict__ grad,
                              float *__restrict__ params, float *__restrict__ m1, float *__restrict__ m2, float lr,
                              float b1c, float b2c, int adam) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k > NPARAM) return;
    float g = 0.0f;
    for (int b = 0; b < nblocks; ++b) g += part[(int64_t)b * (NPARAM + 1) + k];
    grad[k] = g;
    if (!adam || k == NPARAM) return;
    const float a = 0.9f * m1[k] + 0.1f * g;
    const float v = 0.999f * m2[k] + 0.001f * g * g;
    m1[k] = a;
    m2[k] = v;
    params[k] -= lr * (a / b1c) / (sqrtf(v / b2c) + 1e-8f);
}

// feature mean / standard deviation over n samples (one block per feature, fixed order)
__global__ void k_feature_stats(int64_t n, const float *__restrict__ F, float *mu, float *sd) {
    __shared__ double sh[256][2];
    const int f = blockIdx.x;
    double s1 = 0.0, s2 = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        const double x = F[i * NF + f];
        s1 += x;
        s2 += x * x;
    }
    sh[threadIdx.x][0] = s1;
    sh[threadIdx.x][1] = s2;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            sh[threadIdx.x][0] += sh[threadIdx.x + o][0];
            sh[threadIdx.x][1] += sh[threadIdx.x + o][1];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double m = sh[0][0] / (double)n;
        const double v = sh[0][1] / (double)n - m * m;
        mu[f] = (float)m;
        sd[f] = (float)(v > 1e-12 ? sqrt(v) : 1.0);
    }
}

// xhat = T2 e^y; c3 = (xhat - T2)/t^3 -> coef: h [n], then (a, b) pairs [n]; c3 staged in b's slot
// h = xhat = T2 e^y and c3 = (xhat - T2) / t^3, formed as (xhat - T2) times the
// FP64 1/(t*t*t) (t3inv); c3 into c3[i], or with A^2 v into the record
// q[i] = (A^2 v_i, c3_i) of the fused third pass.  t_row / t3inv_row: per-row
// horizons (both, or neither: t_all / t3inv_all).
__global__ void k_cv_xhat(int64_t n, const double *__restrict__ T, const float *__restrict__ y, double t_all,
                          double t3inv_all, const double *__restrict__ t_row, const double *__restrict__ t3inv_row,
                          double *__restrict__ h, double *__restrict__ c3, double2 *__restrict__ q) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double t = t_row ? t_row[i] : t_all;
        const double T2 = T[i] + t * T[n + i] + t * t * T[2 * n + i] / 2.0;
        const double xh = T2 * exp_of_f32(y ? y[i] : 0.0f);
        const double c = (xh - T2) * (t3inv_row ? t3inv_row[i] : t3inv_all);
        h[i] = xh;
        if (q) q[i] = make_double2(T[2 * n + i], c);
        else c3[i] = c;
    }
}

__global__ void k_cv_targets(int64_t n, const double *__restrict__ x, const double *__restrict__ T, double t,
                             float *__restrict__ y) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double T2 = T[i] + t * T[n + i] + t * t * T[2 * n + i] / 2.0;
        const double q = T2 != 0.0 ? x[i] / T2 : 1.0;
        y[i] = (float)log(q > 1e-6 ? q : 1e-6);
    }
}

__global__ void k_cv_ab(int64_t n, const double *__restrict__ T, const double *__restrict__ c3,
                        const double *__restrict__ Ac3, double2 *__restrict__ ab) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        ab[i] = make_double2(T[3 * n + i] / 2.0 - 3.0 * c3[i], Ac3[i]);
}

// ---------------------------------------------------------------------------
// CV walker
// ---------------------------------------------------------------------------
// FP32 residual integrals read the coefficients scaled by 2^-k, k the binary
// exponent of the largest |a_i|, |b_i| (exact), so that the residuals and
// their squares stay inside the FP32 range whatever the scale of v; the means
// and standard errors are scaled back by 2^k when finished.  FP64 integrals
// read them as they are.
struct CVArgs {
    const double *h;        // [n] h(t, i) = xhat_i
    const double2 *ab;      // [n] (a, b) (FP64 integrals)
    const float2 *abf;      // [n] (a, b) 2^-k in FP32 (FP32 integrals, see k_coef_f32)
    const uint32_t *cexp;   // biased exponent word k of the coefficients (FP32 integrals), or NULL
};

__device__ __forceinline__ double coef_scale_up(const CVArgs &cv) { return cv.cexp ? exp_scale(*cv.cexp) : 1.0; }

// the coefficients of state j in the integrals' precision
template <bool F64I>
__device__ __forceinline__ void coef_load(const CVArgs &cv, int32_t j, typename std::conditional<F64I, double, float>::type &ca,
                                          typename std::conditional<F64I, double, float>::type &cb) {
    if constexpr (F64I) {
        const double2 c = __ldg(cv.ab + j);
        ca = c.x;
        cb = c.y;
    } else {
        const float2 c = __ldg(cv.abf + j);
        ca = c.x;
        cb = c.y;
    }
}

__global__ void k_coef_exponent(int64_t n2, const double *__restrict__ ab, uint32_t *word) {
    exponent_max(n2, ab, word);
}

// Residual accumulators: FP64 plain sums, or FP32 per-path scaled sums.
template <bool F64I, bool WEIGHTED>
__global__ void __launch_bounds__(WALK_THREADS) k_walk_cv(const __grid_constant__ WalkParams a, CVArgs cv) {
    using R = typename std::conditional<F64I, double, float>::type;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const uint64_t wid = (uint64_t)blockIdx.x * WARPS_PER_BLOCK + warp;
    const uint64_t n_chunks = (uint64_t)a.n_entries * a.chunks_per_entry;
    if (wid >= n_chunks) return;
    const uint64_t e_idx = wid / a.chunks_per_entry;
    const uint64_t chunk = wid - e_idx * a.chunks_per_entry;
    const int32_t i = a.entries ? __ldg(a.entries + e_idx) : (int32_t)e_idx;
    if (i < 0 || (int64_t)i >= a.n) {
        if (lane == 0) {
            atomicOr(a.status, ST_BAD_ENTRY);
            a.partials[wid] = Partial{QNAN, 0.0, 0.0};
        }
        return;
    }
    const uint64_t p_begin = chunk * a.chunk_len;
    const uint32_t len = (uint32_t)(min(a.paths, p_begin + a.chunk_len) - p_begin);
    const uint64_t base = a.path_offset + p_begin;
    const NodeRec start = load_node(a.node, i);
    Walker<false> w;
    w.rec = start; w.j = i; w.r = a.t32; w.acc = 0.0f; w.delta = start.delta; w.k = 0;
    // per-path residual: y = e^{Ls} ys (FP32) or y (FP64)
    R ys = (R)0;
    float Ls = 0.0f;
    double s1 = 0.0, s2 = 0.0;        // FP64 sums over finished paths (FP64 integral)
    float m = -INFINITY, f1 = 0.f, c1 = 0.f, f2 = 0.f;  // FP32: shifted compensated sums
    uint32_t next = 32, p = (uint32_t)lane;
    bool active = p < len;
    const unsigned lt_mask = (1u << lane) - 1u;
    while (__any_sync(0xffffffffu, active)) {
        bool fin = false;
        if (active) {
            const int32_t j = w.j;
            const float r0 = w.r, L0 = w.acc, dl = w.delta;
            float D;  // the hold just simulated: S (jump) or r0 (end)
            fin = advance<MCX_EXACT, WEIGHTED, false>(w, a, (uint32_t)i, base + p, nullptr, -1, &D);
            R ca, cb;
            coef_load<F64I>(cv, j, ca, cb);
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
            if (fin) {
                if (F64I) {
                    s1 += (double)ys;
                    s2 += (double)ys * (double)ys;
                } else {
                    // fold e^{Ls} ys into the lane's shifted compensated sums
                    const float Lp = Ls;
                    if (!(Lp <= m + 8.0f)) {
                        const float sc = (m == -INFINITY) ? 0.0f : expf(m - Lp);
                        f1 *= sc; c1 *= sc; f2 *= sc * sc;
                        m = Lp;
                    }
                    const float wv = __fmul_rn(expf(__fsub_rn(Lp, m)), (float)ys);
                    const float yk = __fsub_rn(wv, c1);
                    const float tk = __fadd_rn(f1, yk);
                    c1 = __fsub_rn(__fsub_rn(tk, f1), yk);
                    f1 = tk;
                    f2 = __fmaf_rn(wv, wv, f2);
                }
            }
        }
        const unsigned fm = __ballot_sync(0xffffffffu, fin);
        if (fm) {
            if (fin) {
                p = next + (uint32_t)__popc(fm & lt_mask);
                active = p < len;
                w.rec = start; w.j = i; w.r = a.t32; w.acc = 0.0f; w.delta = start.delta; w.k = 0;
                ys = (R)0;
                Ls = 0.0f;
            }
            next += (uint32_t)__popc(fm);
        }
    }
    double S1, S2, Mw;
    if (F64I) {
        S1 = s1;
        S2 = s2;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            S1 += __shfl_xor_sync(0xffffffffu, S1, o);
            S2 += __shfl_xor_sync(0xffffffffu, S2, o);
        }
        Mw = 0.0;
    } else {
        float mw = m;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mw = fmaxf(mw, __shfl_xor_sync(0xffffffffu, mw, o));
        const double sc = (m == -INFINITY) ? 0.0 : exp((double)m - (double)mw);
        S1 = sc * ((double)f1 - (double)c1);
        S2 = sc * sc * (double)f2;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            S1 += __shfl_xor_sync(0xffffffffu, S1, o);
            S2 += __shfl_xor_sync(0xffffffffu, S2, o);
        }
        Mw = (double)mw;
    }
    if (lane == 0) a.partials[wid] = Partial{S1, S2, Mw};
}

// Few paths per entry: one lane per entry, paths in path order, the lane writes
// the entry's result (no partials).
template <bool F64I, bool WEIGHTED>
__global__ void __launch_bounds__(WALK_THREADS) k_walk_cv_lanes(const __grid_constant__ WalkParams a, CVArgs cv) {
    using R = typename std::conditional<F64I, double, float>::type;
    const int64_t e = (int64_t)blockIdx.x * WALK_THREADS + threadIdx.x;
    const bool valid = e < a.n_entries;
    unsigned long long jumps = 0, npaths = 0;
    if (valid) {
        const int32_t i = a.entries ? __ldg(a.entries + e) : (int32_t)e;
        if (i < 0 || (int64_t)i >= a.n) {
            atomicOr(a.status, ST_BAD_ENTRY);
            a.mean[e] = QNAN;
            if (a.sem) a.sem[e] = QNAN;
        } else {
            const NodeRec start = load_node(a.node, i);
            double s1 = 0.0, s2 = 0.0;                           // FP64 residual sums
            float m = -INFINITY, f1 = 0.f, c1 = 0.f, f2 = 0.f;  // FP32 shifted sums
            for (uint64_t p = 0; p < a.paths; ++p) {
                Walker<false> w;
                w.rec = start; w.j = i; w.r = a.t32; w.acc = 0.0f; w.delta = start.delta; w.k = 0;
                R ys = (R)0;
                float Ls = 0.0f;
                bool fin = false;
                while (!fin) {
                    const int32_t j = w.j;
                    const float r0 = w.r, L0 = w.acc, dl = w.delta;
                    float D;
                    fin = advance<MCX_EXACT, WEIGHTED, false>(w, a, (uint32_t)i, a.path_offset + p, nullptr, -1, &D);
                    R ca, cb;
                    coef_load<F64I>(cv, j, ca, cb);
                    const R J = hold_integral<R>(ca, cb, (R)dl, (R)r0, (R)D);
                    if (F64I) {
                        ys += (R)exp((double)L0) * J;
                    } else {
                        if (L0 > Ls + 40.0f) {
                            ys *= (R)expf(Ls - L0);
                            Ls = L0;
                        }
                        ys += (R)expf(L0 - Ls) * J;
                    }
                }
                jumps += w.k;
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
            npaths = a.paths;
            if (!F64I && m <= 80.0f) {
                // the residual is a correction to h: its mean and standard error in FP32
                // (M <= 64 here, exact), added to h in FP64
                const float M = (float)a.paths;
                const float S1 = __fsub_rn(f1, c1);
                const float sc = expf(m);
                const float mu = __fdiv_rn(S1, M);
                float var = M > 1.0f ? __fdiv_rn(__fsub_rn(f2, __fmul_rn(S1, mu)), M - 1.0f) : 0.0f;
                if (var < 0.0f) var = 0.0f;
                const double up = coef_scale_up(cv);  // undo the coefficients' power-of-two scaling
                a.mean[e] = cv.h[i] + (double)__fmul_rn(sc, mu) * up;
                if (a.sem) a.sem[e] = (double)__fmul_rn(sc, sqrtf(__fdiv_rn(var, M))) * up;
            } else {
                double S1, S2, scale;
                if (F64I) {
                    S1 = s1;
                    S2 = s2;
                    scale = 1.0;
                } else {
                    S1 = (double)f1 - (double)c1;
                    S2 = (double)f2;
                    scale = exp((double)m) * coef_scale_up(cv);
                }
                const double M = (double)a.paths;
                const double mu = S1 / M;
                double var = M > 1.0 ? (S2 - S1 * mu) / (M - 1.0) : 0.0;
                if (var < 0.0) var = 0.0;
                a.mean[e] = cv.h[i] + scale * mu;
                if (a.sem) a.sem[e] = scale * sqrt(var / M);
            }
            if (!isfinite(a.mean[e])) atomicOr(a.status, ST_OVERFLOW);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        jumps += __shfl_xor_sync(0xffffffffu, jumps, o);
        npaths += __shfl_xor_sync(0xffffffffu, npaths, o);
    }
    if ((threadIdx.x & 31) == 0 && npaths) {
        unsigned long long *ctr = reinterpret_cast<unsigned long long *>(a.status + 2);
        atomicAdd(ctr, npaths);
        atomicAdd(ctr + 1, jumps);
    }
}

// mean = h_i + (e^m sum y)/M over the entry's chunks; sem from the residual variance
__global__ void k_cv_finish(const Partial *__restrict__ part, int64_t n_entries, uint32_t cpe, double M,
                            const int32_t *__restrict__ entries, const double *__restrict__ h,
                            const uint32_t *__restrict__ cexp, double *mean, double *sem, uint32_t *status) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_entries) return;
    const Partial *pp = part + (uint64_t)e * cpe;
    double mx = -INFINITY;
    for (uint32_t c = 0; c < cpe; ++c) mx = fmax(mx, pp[c].m);
    double s1 = 0.0, s2 = 0.0;
    bool bad = false;
    for (uint32_t c = 0; c < cpe; ++c) {
        const Partial q = pp[c];
        if (isnan(q.s1)) bad = true;
        const double sc = q.m == -INFINITY ? 0.0 : exp(q.m - mx);
        s1 += sc * q.s1;
        s2 += sc * sc * q.s2;
    }
    const int64_t i = entries ? entries[e] : e;
    if (bad) {
        mean[e] = QNAN;
        if (sem) sem[e] = QNAN;
        return;
    }
    const double scale = (mx == -INFINITY ? 0.0 : exp(mx)) * (cexp ? exp_scale(*cexp) : 1.0);
    const double mu = s1 / M;
    double var = M > 1.0 ? (s2 - s1 * mu) / (M - 1.0) : 0.0;
    if (var < 0.0) var = 0.0;
    mean[e] = h[i] + scale * mu;
    if (sem) sem[e] = scale * sqrt(var / M);
    if (!isfinite(mean[e])) atomicOr(status, ST_OVERFLOW);
}

unsigned blocks_for(int64_t n, int threads) {
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + threads - 1) / threads, 152 * 32));
}

}  // namespace

// A row schedule carved from float64 scratch at `w`: order [n] int32, then the
// counters and the window starts.
void carve_schedule(int64_t n, double *w, CvRowSchedule &s) {
    s.order = reinterpret_cast<int32_t *>(w);
    s.cnt = reinterpret_cast<uint32_t *>(w) + n;
    s.hist = s.cnt + CV_ROW_CNT;
}

// Taylor terms v, Av, A^2 v (and A^3 v when `third`) and the features of rows
// 0..n-1 (see mcx_cv_prepare) in two row passes (three with `third`); t_row,
// when given, holds each row's own horizon (rows of several problems at once).
// s: the rows' schedule; ell: its short rows' sliced ELL copy or NULL; g: [n]
// records, 16-byte aligned; lam: float64 [n] scratch (may be taylor + 3n when
// `third`: the third pass overwrites it).
cudaError_t cv_taylor_rows(int64_t n, const int64_t *row_ptr, const int32_t *col, const double *val,
                           const double *v, double t, const double *t_row, const CvRowSchedule &s, const CvSell *ell,
                           double2 *g, double *lam, double *taylor, float *features, bool third, cudaStream_t st) {
    const cudaError_t e = cudaMemcpyAsync(taylor, v, sizeof(double) * (size_t)n, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return e;
    run_pass(row_ptr, col, val, s, ell, PassRates{row_ptr, col, val, v, taylor + n, lam, g}, st);
    run_pass(row_ptr, col, val, s, ell,
             PassFeatures{row_ptr, col, val, g, v, lam, taylor + 2 * n, features, t, t_row}, st);
    if (third) run_pass(row_ptr, col, val, s, ell, PassSpmv{taylor + 2 * n, taylor + 3 * n}, st);
    return cudaGetLastError();
}

// mcx_cv_prepare; work: float64 [3n + 64], 16-byte aligned.
cudaError_t cv_prepare_rows(int64_t n, const int64_t *row_ptr, const int32_t *col, const double *val,
                            const double *v, double t, double *work, double *taylor, float *features,
                            cudaStream_t st) {
    double2 *g = reinterpret_cast<double2 *>(work);  // 2n doubles
    CvRowSchedule s;
    carve_schedule(n, work + 2 * n, s);
    const cudaError_t e = build_schedule(n, row_ptr, s, st);
    if (e != cudaSuccess) return e;
    return cv_taylor_rows(n, row_ptr, col, val, v, t, nullptr, s, nullptr, g, taylor + 3 * n, taylor, features,
                          true, st);
}

// mcx_cv_coefficients into ab [n] and h [n]; work: float64 [3n + 64].
cudaError_t cv_coefficients_rows(int64_t n, const int64_t *row_ptr, const int32_t *col, const double *val,
                                 const double *taylor, const float *y, double t, double *work, double2 *ab,
                                 double *h, cudaStream_t st) {
    const unsigned nb = blocks_for(n, 256);
    double *c3 = work, *Ac3 = work + n;
    CvRowSchedule s;
    carve_schedule(n, work + 2 * n, s);
    const cudaError_t e = build_schedule(n, row_ptr, s, st);
    if (e != cudaSuccess) return e;
    k_cv_xhat<<<nb, 256, 0, st>>>(n, taylor, y, t, 1.0 / (t * t * t), nullptr, nullptr, h, c3, nullptr);
    run_pass(row_ptr, col, val, s, nullptr, PassSpmv{c3, Ac3}, st);
    k_cv_ab<<<nb, 256, 0, st>>>(n, taylor, c3, Ac3, ab);
    return cudaGetLastError();
}

// The same coefficients from the Taylor terms v, Av, A^2 v alone: A^3 v and A c3
// in one row pass over the records (A^2 v_c, c3_c) (q: [n], 16-byte aligned);
// bit-identical to cv_prepare_rows' A^3 v followed by cv_coefficients_rows.
cudaError_t cv_cubic_rows(int64_t n, const int64_t *row_ptr, const int32_t *col, const double *val,
                          const double *taylor, const float *y, const double *t_row, const double *t3inv_row,
                          const CvRowSchedule &s, const CvSell *ell, double2 *q, double2 *ab, double *h,
                          cudaStream_t st) {
    k_cv_xhat<<<blocks_for(n, 256), 256, 0, st>>>(n, taylor, y, 0.0, 0.0, t_row, t3inv_row, h, nullptr, q);
    run_pass(row_ptr, col, val, s, ell, PassCubic{q, ab}, st);
    return cudaGetLastError();
}

}  // namespace mcx

using namespace mcx;

struct mcx_mlp {
    float *params = nullptr;  // [NPARAM + 1] (last: unused)
    float *m1 = nullptr, *m2 = nullptr;
    float *stats = nullptr;   // mu [NF], sd [NF]
    float *grad = nullptr;    // [NPARAM + 1] (last: loss)
    float *part = nullptr;
    int64_t part_blocks = 0;
    float *losses = nullptr;  // per-minibatch losses of one epoch (device)
    int64_t losses_n = 0;
    int64_t *idx = nullptr;   // minibatch permutation
    int64_t idx_n = 0;
    int64_t step = 0;
    uint32_t *err = nullptr;  // latched device status of inference (bit 0: an MMA wait gave up)
    uint32_t wait_polls = TC_WAIT;  // polls of the MMA completion wait (test hook: mcx_debug_mlp_wait_polls)
};

namespace {

mcx_status cv_status(cudaError_t e) {
    if (e == cudaSuccess) return MCX_OK;
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return MCX_E_OOM;
    }
    return MCX_E_CUDA;
}

MLPView view(const mcx_mlp *m) { return MLPView{m->params, m->stats, m->stats + NF}; }

cudaError_t ensure_part(mcx_mlp *m, int64_t blocks) {
    if (m->part_blocks >= blocks) return cudaSuccess;
    dev_free(m->part);
    m->part = nullptr;
    m->part_blocks = 0;
    cudaError_t e = dev_malloc(&m->part, sizeof(float) * (NPARAM + 1) * (size_t)blocks);
    if (e == cudaSuccess) m->part_blocks = blocks;
    return e;
}


}  // namespace

extern "C" {

mcx_status mcx_cv_prepare(int64_t n, const int64_t *row_ptr, const int32_t *col, const double *val, const double *v,
                          double t, double *work, double *taylor, float *features, void *stream) {
    NvtxRange nvtx("mcx_cv_prepare");
    if (n < 1 || !row_ptr || !col || !val || !v || !work || !taylor || !features || !(t > 0.0)) return MCX_E_INVALID;
    if (reinterpret_cast<uintptr_t>(work) & 15u) return MCX_E_INVALID;  // 16-byte records
    return cv_status(cv_prepare_rows(n, row_ptr, col, val, v, t, work, taylor, features,
                                     static_cast<cudaStream_t>(stream)));
}

mcx_status mcx_cv_targets(int64_t n, const double *x, const double *taylor, double t, float *y, void *stream) {
    if (n < 1 || !x || !taylor || !y || !(t > 0.0)) return MCX_E_INVALID;
    k_cv_targets<<<blocks_for(n, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(n, x, taylor, t, y);
    return cv_status(cudaGetLastError());
}

mcx_status mcx_mlp_create(uint64_t seed, mcx_mlp **out) {
    if (!out) return MCX_E_INVALID;
    *out = nullptr;
    mcx_mlp *m = new (std::nothrow) mcx_mlp();
    if (!m) return MCX_E_OOM;
    // He-uniform weights from a counter-based stream (host), small uniform biases
    std::vector<float> p(NPARAM + 1, 0.0f);
    uint64_t s = seed * 0x9E3779B97F4A7C15ull + 0x2545F4914F6CDD1Dull;
    auto unif = [&s]() {  // splitmix64
        s += 0x9E3779B97F4A7C15ull;
        uint64_t z = s;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        return (double)(z >> 11) * 0x1p-53;
    };
    auto fill = [&](int off, int count, double lim) {
        for (int k = 0; k < count; ++k) p[off + k] = (float)((2.0 * unif() - 1.0) * lim);
    };
    fill(P_W1, NF * HID, sqrt(6.0 / NF));
    fill(P_B1, HID, 0.1);
    fill(P_W2, HID * HID, sqrt(6.0 / HID));
    fill(P_B2, HID, 0.1);
    fill(P_W3, HID, sqrt(6.0 / HID) * 0.1);
    p[P_B3] = 0.0f;
    std::vector<float> stats(2 * NF, 0.0f);
    for (int f = 0; f < NF; ++f) stats[NF + f] = 1.0f;
    cudaError_t e;
    do {
        if ((e = dev_malloc(&m->params, sizeof(float) * (NPARAM + 1))) != cudaSuccess) break;
        if ((e = dev_malloc(&m->m1, sizeof(float) * (NPARAM + 1))) != cudaSuccess) break;
        if ((e = dev_malloc(&m->m2, sizeof(float) * (NPARAM + 1))) != cudaSuccess) break;
        if ((e = dev_malloc(&m->grad, sizeof(float) * (NPARAM + 1))) != cudaSuccess) break;
        if ((e = dev_malloc(&m->stats, sizeof(float) * 2 * NF)) != cudaSuccess) break;
        if ((e = dev_malloc(&m->err, sizeof(uint32_t))) != cudaSuccess) break;
        cudaMemset(m->err, 0, sizeof(uint32_t));
        cudaMemcpy(m->params, p.data(), sizeof(float) * (NPARAM + 1), cudaMemcpyHostToDevice);
        cudaMemcpy(m->stats, stats.data(), sizeof(float) * 2 * NF, cudaMemcpyHostToDevice);
        cudaMemset(m->m1, 0, sizeof(float) * (NPARAM + 1));
        e = cudaMemset(m->m2, 0, sizeof(float) * (NPARAM + 1));
    } while (0);
    if (e != cudaSuccess) {
        mcx_mlp_destroy(m);
        return cv_status(e);
    }
    *out = m;
    return MCX_OK;
}

mcx_status mcx_mlp_set(mcx_mlp *m, const float *params, const float *mu, const float *sd) {
    if (!m) return MCX_E_INVALID;
    cudaError_t e = cudaSuccess;
    if (params) e = cudaMemcpy(m->params, params, sizeof(float) * NPARAM, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && mu) e = cudaMemcpy(m->stats, mu, sizeof(float) * NF, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && sd) e = cudaMemcpy(m->stats + NF, sd, sizeof(float) * NF, cudaMemcpyHostToDevice);
    return cv_status(e);
}

mcx_status mcx_mlp_get(const mcx_mlp *m, float *params, float *mu, float *sd) {
    if (!m) return MCX_E_INVALID;
    cudaError_t e = cudaSuccess;
    if (params) e = cudaMemcpy(params, m->params, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && mu) e = cudaMemcpy(mu, m->stats, sizeof(float) * NF, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && sd) e = cudaMemcpy(sd, m->stats + NF, sizeof(float) * NF, cudaMemcpyDeviceToHost);
    return cv_status(e);
}

mcx_status mcx_mlp_predict(const mcx_mlp *m, int64_t n, const float *features, float *y, void *stream) {
    NvtxRange nvtx("mcx_mlp_predict");
    if (!m || n < 0 || (n > 0 && (!features || !y))) return MCX_E_INVALID;
    if (n == 0) return MCX_OK;
    const int64_t tiles = (n + TC_ROWS - 1) / TC_ROWS;
    // 7 resident CTAs per SM (registers and shared memory allow 7; 7 x 64 of the 512 TMEM columns)
    const unsigned grid = (unsigned)std::min<int64_t>(tiles, 152 * 7);
    k_mlp_predict_tc<<<grid, TC_ROWS, 0, static_cast<cudaStream_t>(stream)>>>(n, features, view(m), y, m->err,
                                                                              m->wait_polls);
    return cv_status(cudaGetLastError());
}

mcx_status mcx_debug_mlp_wait_polls(mcx_mlp *m, uint32_t polls) {
    if (!m) return MCX_E_INVALID;
    m->wait_polls = polls == 0xFFFFFFFFu ? TC_WAIT : polls;
    return MCX_OK;
}

mcx_status mcx_mlp_sync(mcx_mlp *m, void *stream) {
    if (!m) return MCX_E_INVALID;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    uint32_t h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, m->err, sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess && h) e = cudaMemsetAsync(m->err, 0, sizeof(uint32_t), st);
    if (e != cudaSuccess) return cv_status(e);
    return h ? MCX_E_TIMEOUT : MCX_OK;
}

mcx_status mcx_mlp_gradient(mcx_mlp *m, int64_t n, const float *features, const float *targets, float *grad,
                            float *loss, void *stream) {
    NvtxRange nvtx("mcx_mlp_gradient");
    if (!m || n < 1 || !features || !targets || !grad) return MCX_E_INVALID;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int64_t blocks = (n + TG_ROWS - 1) / TG_ROWS;
    cudaError_t e = ensure_part(m, blocks);
    if (e != cudaSuccess) return cv_status(e);
    cudaFuncSetAttribute(k_mlp_grad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TG_SMEM);
    k_mlp_grad_tc<<<(unsigned)blocks, TG_ROWS, TG_SMEM, st>>>(n, features, targets, nullptr, view(m),
                                                               1.0f / (float)n, m->part, m->err, m->wait_polls);
    k_grad_reduce<<<(NPARAM + 256) / 256, 256, 0, st>>>((int)blocks, m->part, m->grad, nullptr, nullptr, nullptr,
                                                         0.f, 1.f, 1.f, 0);
    e = cudaMemcpyAsync(grad, m->grad, sizeof(float) * NPARAM, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess && loss) {
        e = cudaMemcpyAsync(loss, m->grad + NPARAM, sizeof(float), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    return cv_status(e == cudaSuccess ? cudaGetLastError() : e);
}

mcx_status mcx_mlp_fit(mcx_mlp *m, int64_t n, const float *features, const float *targets, int32_t epochs,
                       int32_t batch, float lr, uint64_t seed, float *epoch_loss, void *stream) {
    NvtxRange nvtx("mcx_mlp_fit");
    if (!m || n < 1 || !features || !targets || epochs < 0 || batch < 1 || !(lr > 0.0f)) return MCX_E_INVALID;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // feature standardisation from this training set
    k_feature_stats<<<NF, 256, 0, st>>>(n, features, m->stats, m->stats + NF);
    const int64_t bblocks = (batch + TG_ROWS - 1) / TG_ROWS;
    cudaError_t e = ensure_part(m, bblocks);
    if (e != cudaSuccess) return cv_status(e);
    if (m->idx_n < n) {
        dev_free(m->idx);
        m->idx = nullptr;
        if ((e = dev_malloc(&m->idx, sizeof(int64_t) * (size_t)n)) != cudaSuccess) return cv_status(e);
        m->idx_n = n;
    }
    const int64_t steps = (n + batch - 1) / batch;  // minibatches per epoch
    if (epoch_loss && m->losses_n < steps) {
        dev_free(m->losses);
        m->losses = nullptr;
        if ((e = dev_malloc(&m->losses, sizeof(float) * (size_t)steps)) != cudaSuccess) return cv_status(e);
        m->losses_n = steps;
    }
    cudaFuncSetAttribute(k_mlp_grad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TG_SMEM);
    std::vector<int64_t> perm(n);
    std::vector<float> hl(epoch_loss ? (size_t)steps : 0);
    uint64_t s = seed * 0xD1B54A32D192ED03ull + 1;
    for (int32_t ep = 0; ep < epochs; ++ep) {
        for (int64_t i = 0; i < n; ++i) perm[i] = i;
        for (int64_t i = n - 1; i > 0; --i) {  // Fisher-Yates with splitmix64
            s += 0x9E3779B97F4A7C15ull;
            uint64_t z = s;
            z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
            z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
            z ^= z >> 31;
            std::swap(perm[i], perm[(int64_t)(z % (uint64_t)(i + 1))]);
        }
        cudaMemcpyAsync(m->idx, perm.data(), sizeof(int64_t) * (size_t)n, cudaMemcpyHostToDevice, st);
        double eloss = 0.0;
        int64_t nb = 0;
        for (int64_t b0 = 0; b0 < n; b0 += batch) {
            const int64_t bn = std::min<int64_t>(batch, n - b0);
            const int64_t blocks = (bn + TG_ROWS - 1) / TG_ROWS;
            ++m->step;
            const float b1c = 1.0f - powf(0.9f, (float)m->step);
            const float b2c = 1.0f - powf(0.999f, (float)m->step);
            k_mlp_grad_tc<<<(unsigned)blocks, TG_ROWS, TG_SMEM, st>>>(bn, features, targets, m->idx + b0, view(m),
                                                                       1.0f / (float)bn, m->part, m->err,
                                                                       m->wait_polls);
            k_grad_reduce<<<(NPARAM + 256) / 256, 256, 0, st>>>((int)blocks, m->part, m->grad, m->params, m->m1,
                                                                 m->m2, lr, b1c, b2c, 1);
            if (epoch_loss)  // kept on the device; read once per epoch
                cudaMemcpyAsync(m->losses + nb, m->grad + NPARAM, sizeof(float), cudaMemcpyDeviceToDevice, st);
            ++nb;
        }
        if (epoch_loss) {
            if ((e = cudaMemcpyAsync(hl.data(), m->losses, sizeof(float) * (size_t)nb, cudaMemcpyDeviceToHost, st)) !=
                    cudaSuccess ||
                (e = cudaStreamSynchronize(st)) != cudaSuccess)
                return cv_status(e);
            for (int64_t k = 0; k < nb; ++k) eloss += hl[k];
            epoch_loss[ep] = (float)(eloss / (double)std::max<int64_t>(nb, 1));
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return cv_status(e);
    }
    return cv_status(cudaStreamSynchronize(st));
}

void mcx_mlp_destroy(mcx_mlp *m) {
    if (!m) return;
    dev_free(m->params);
    dev_free(m->m1);
    dev_free(m->m2);
    dev_free(m->stats);
    dev_free(m->grad);
    dev_free(m->part);
    dev_free(m->idx);
    dev_free(m->err);
    dev_free(m->losses);
    delete m;
}

mcx_status mcx_cv_coefficients(int64_t n, const int64_t *row_ptr, const int32_t *col, const double *val,
                               const double *taylor, const float *y, double t, double *work, double *coef,
                               void *stream) {
    NvtxRange nvtx("mcx_cv_coefficients");
    if (n < 1 || !row_ptr || !col || !val || !taylor || !work || !coef || !(t > 0.0)) return MCX_E_INVALID;
    if (reinterpret_cast<uintptr_t>(coef) % 16 != 0) return MCX_E_INVALID;
    // layout: (a, b) pairs at offset 0 (16-byte aligned with the buffer), then h
    return cv_status(cv_coefficients_rows(n, row_ptr, col, val, taylor, y, t, work,
                                          reinterpret_cast<double2 *>(coef), coef + 2 * n,
                                          static_cast<cudaStream_t>(stream)));
}

mcx_status mcx_estimate_cv(mcx_plan *plan, const double *coef, double t, uint64_t paths, const int32_t *entries,
                           int64_t n_entries, uint64_t seed, uint64_t path_offset, int precision, double *mean,
                           double *sem, void *stream) {
    NvtxRange nvtx("mcx_estimate_cv");
    if (!plan || !coef || !(t > 0.0) || !isfinite(t) || paths < 1 || paths > (1ull << 53)) return MCX_E_INVALID;
    if (precision != MCX_FP32 && precision != MCX_FP64) return MCX_E_INVALID;
    if (n_entries == 0) return MCX_OK;
    if (n_entries < 0 || !mean || (!entries && n_entries != plan->n)) return MCX_E_INVALID;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    WalkParams p{};
    p.node = plan->node;
    p.node64 = plan->node64;
    p.edge_col = plan->edge_col;
    p.edge16 = plan->edge16;
    p.entries = entries;
    p.n_entries = n_entries;
    p.paths = paths;
    p.nsteps = 1;
    p.n = plan->n;
    p.max_events = 1u << 30;
    p.t64 = t;
    p.t32 = (float)t;
    p.path_offset = path_offset;
    p.status = plan->status;
    set_round_keys(p, seed);
    if (reinterpret_cast<uintptr_t>(coef) % 16 != 0) return MCX_E_INVALID;  // (a, b) pairs are read as double2
    const bool wgt = plan->weighted_rows > 0;
    const uint32_t *cexp = nullptr;  // FP32 integrals: the coefficients' exponent, for their scaling
    float2 *abf = nullptr;           // FP32 integrals: their scaled FP32 copy (pool, freed after the walk)
    if (precision == MCX_FP32) {
        uint32_t *word = plan->status + STATUS_CEXP;
        cudaError_t e0 = cudaMemsetAsync(word, 0, sizeof(uint32_t), st);
        if (e0 == cudaSuccess) e0 = pool_alloc(reinterpret_cast<void **>(&abf), sizeof(float2) * (size_t)plan->n, st);
        if (e0 != cudaSuccess) return cv_status(e0);
        k_coef_exponent<<<blocks_for(2 * plan->n, 256), 256, 0, st>>>(2 * plan->n, coef, word);
        k_coef_f32<<<blocks_for(plan->n, 256), 256, 0, st>>>(plan->n, reinterpret_cast<const double2 *>(coef), word,
                                                             abf);
        cexp = word;
    }
    struct PoolRelease {  // the FP32 copy goes back to the pool behind the walk on the stream
        float2 *p;
        cudaStream_t s;
        ~PoolRelease() { pool_free(p, s); }
    } release{abf, st};
    if (paths <= LANE_MODE_MAX_PATHS) {  // few paths per entry: one lane per entry
        p.mean = mean;
        p.sem = sem;
        CVArgs cvl{coef + 2 * plan->n, reinterpret_cast<const double2 *>(coef), abf, cexp};
        const unsigned grid = (unsigned)((n_entries + WALK_THREADS - 1) / WALK_THREADS);
        if (precision == MCX_FP64) {
            if (wgt) k_walk_cv_lanes<true, true><<<grid, WALK_THREADS, 0, st>>>(p, cvl);
            else k_walk_cv_lanes<true, false><<<grid, WALK_THREADS, 0, st>>>(p, cvl);
        } else {
            if (wgt) k_walk_cv_lanes<false, true><<<grid, WALK_THREADS, 0, st>>>(p, cvl);
            else k_walk_cv_lanes<false, false><<<grid, WALK_THREADS, 0, st>>>(p, cvl);
        }
        return cv_status(cudaGetLastError());
    }
    const uint64_t target_warps = 152ull * 64ull * 8ull;
    uint64_t cpe = (target_warps + (uint64_t)n_entries - 1) / (uint64_t)n_entries;
    const uint64_t max_cpe = (paths + 1023) / 1024;
    if (cpe > max_cpe) cpe = max_cpe;
    if (cpe < 1) cpe = 1;
    if ((paths + cpe - 1) / cpe > (1ull << 30)) cpe = (paths + (1ull << 30) - 1) >> 30;
    uint64_t chunk = (paths + cpe - 1) / cpe;
    chunk = (chunk + 31) / 32 * 32;
    cpe = (paths + chunk - 1) / chunk;
    p.chunk_len = chunk;
    p.chunks_per_entry = (uint32_t)cpe;
    const uint64_t n_chunks = (uint64_t)n_entries * cpe;
    const size_t need = sizeof(Partial) * (size_t)n_chunks;
    if (plan->scratch_bytes < need) {
        dev_free(plan->scratch);
        plan->scratch = nullptr;
        plan->scratch_bytes = 0;
        cudaError_t e = dev_malloc(&plan->scratch, need);
        if (e != cudaSuccess) return cv_status(e);
        plan->scratch_bytes = need;
    }
    p.partials = static_cast<Partial *>(plan->scratch);
    CVArgs cv{coef + 2 * plan->n, reinterpret_cast<const double2 *>(coef), abf, cexp};
    const unsigned grid = (unsigned)((n_chunks + WARPS_PER_BLOCK - 1) / WARPS_PER_BLOCK);
    if (precision == MCX_FP64) {
        if (wgt) k_walk_cv<true, true><<<grid, WALK_THREADS, 0, st>>>(p, cv);
        else k_walk_cv<true, false><<<grid, WALK_THREADS, 0, st>>>(p, cv);
    } else {
        if (wgt) k_walk_cv<false, true><<<grid, WALK_THREADS, 0, st>>>(p, cv);
        else k_walk_cv<false, false><<<grid, WALK_THREADS, 0, st>>>(p, cv);
    }
    k_cv_finish<<<(unsigned)((n_entries + 255) / 256), 256, 0, st>>>(p.partials, n_entries, (uint32_t)cpe,
                                                                       (double)paths, entries, coef + 2 * plan->n,
                                                                       cexp, mean, sem, plan->status);
    return cv_status(cudaGetLastError());
}

}  // extern "C"
