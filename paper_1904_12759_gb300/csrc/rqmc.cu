// Randomised quasi-Monte Carlo backward estimator (a variance-reduction
// direction named in Sec. 5).
//
// The first QMC_EVENTS events of every path take their holding-time word
// (word 0) and slot word (word 2) from a scrambled Sobol' point instead of the
// path's Philox block: event k reads dimensions 2k and 2k + 1.  Words 1 and 3
// and every later event keep the path's Philox draws, with path index
// r 2^m + q for point q of replicate r.  Everything else (holding times, the
// stop rule, the jump tables, the three functionals) is the walker of
// walker.cuh unchanged, so each path is still an exact sample of the chain.
//
// Sobol' points (Sobol' 1967; Bratley & Fox 1988): coordinate d of point q is
// the XOR of direction numbers V_d[b] over the set bits b of q.  Dimension 0 is
// van der Corput's (V_0[b] = 2^(31-b)); dimension d >= 1 has a primitive
// polynomial x^s + a_1 x^(s-1) + ... + a_(s-1) x + 1 over GF(2) and initial odd
// m_1..m_s, continued by m_k = (XOR_c a_c 2^c m_(k-c)) ^ 2^s m_(k-s) ^ m_(k-s),
// V_d[k-1] = m_k 2^(32-k).  The parameters are the first entries of Joe & Kuo's
// table (2003, 2008).
//
// Randomisation per replicate (Matousek 1998): a random lower-triangular
// binary matrix L_(r,d) with unit diagonal (output bit b, counted from the most
// significant, mixes input bits 0..b) scrambles the direction numbers, and a
// random digital shift e_(i,r,d) is XORed per entry.  Nets stay nets and every
// point is uniform, so each replicate mean is unbiased; the spread of the R
// independent replicate means gives the standard error.  Row b of L_(r,d) is
// word 0 of Philox {b, 0xFFFFFFFC, d, r} (bits above b kept, bit b set);
// e_(i,r,d) is word d mod 4 of Philox {d / 4, 0xFFFFFFFD, i, r}.
//
// Work decomposition: a setup kernel turns each replicate's scrambled
// direction numbers into digit tables (global memory, shared by all entries),
// so a coordinate costs one load per 5 bits of the point index.  Then one warp
// per (entry, group of replicates, slice).  With many entries a warp takes all
// replicates of one entry, stages the entry row once, folds the replicate
// means itself and the last warp of each block finishes the block's entries;
// with few entries a replicate's 2^m points are cut into slices over several
// warps, each writing one log-shifted partial sum per (replicate, slice) that
// k_rqmc_finish merges into replicate means and then into the estimate and its
// standard error.
#include <math.h>

#include <type_traits>

#include "accum.cuh"
#include "launch.h"
#include "walker.cuh"

namespace mcx {
namespace {

constexpr int QMC_DIMS = MCX_QMC_DIMS;
constexpr uint32_t QMC_EVENTS = QMC_DIMS / 2;
constexpr uint32_t STREAM_SCRAMBLE = 0xFFFFFFFCu;
constexpr uint32_t STREAM_SHIFT = 0xFFFFFFFDu;

// Degree, coefficient bits a_1..a_(s-1) (a_1 the most significant) and
// m_1..m_s of dimensions 1..15.
struct SobolInit {
    int s;
    uint32_t a;
    uint32_t m[6];
};
constexpr SobolInit kSobolInit[QMC_DIMS - 1] = {
    {1, 0u, {1}},
    {2, 1u, {1, 3}},
    {3, 1u, {1, 3, 1}},
    {3, 2u, {1, 1, 1}},
    {4, 1u, {1, 1, 3, 3}},
    {4, 4u, {1, 3, 5, 13}},
    {5, 2u, {1, 1, 5, 5, 17}},
    {5, 4u, {1, 1, 5, 5, 5}},
    {5, 7u, {1, 1, 7, 11, 19}},
    {5, 11u, {1, 1, 5, 1, 1}},
    {5, 13u, {1, 1, 1, 3, 11}},
    {5, 14u, {1, 3, 5, 5, 31}},
    {6, 1u, {1, 3, 3, 9, 7, 49}},
    {6, 13u, {1, 1, 1, 15, 21, 21}},
    {6, 16u, {1, 3, 1, 13, 27, 49}},
};

struct SobolBase {
    uint32_t v[QMC_DIMS][32];
};

// Unscrambled direction numbers (host).
SobolBase sobol_base() {
    SobolBase B{};
    for (int b = 0; b < 32; ++b) B.v[0][b] = 0x80000000u >> b;
    for (int d = 1; d < QMC_DIMS; ++d) {
        const SobolInit &P = kSobolInit[d - 1];
        uint64_t m[33] = {0};
        for (int k = 1; k <= 32; ++k) {
            if (k <= P.s) {
                m[k] = P.m[k - 1];
            } else {
                uint64_t x = m[k - P.s] ^ (m[k - P.s] << P.s);
                for (int c = 1; c < P.s; ++c) {
                    const uint32_t a_c = (P.a >> (P.s - 1 - c)) & 1u;
                    if (a_c) x ^= m[k - c] << c;
                }
                m[k] = x;
            }
            B.v[d][k - 1] = (uint32_t)(m[k] << (32 - k));
        }
    }
    return B;
}

// Coordinates are read from per-replicate digit tables: the index q is cut
// into 5-bit digits, and table level l of dimension d holds, for each digit
// value c, the XOR of the scrambled direction numbers of the bits set in c at
// positions 5l .. 5l+4.  A coordinate is then the XOR of one entry per level
// (ceil(log2q / 5) loads, no branches).
constexpr uint32_t QMC_DIGIT = 5;
constexpr uint32_t QMC_LEVELS = (MCX_QMC_MAX_LOG2 + QMC_DIGIT - 1) / QMC_DIGIT;

// One thread per (replicate r0 + r, dimension d): the scrambled direction
// numbers L_(r0+r,d) V_d[b], b < bits, then the digit tables
// tabs[((r * QMC_DIMS + d) * nlev + l) * 32 + c].
__global__ void k_qmc_scramble(const __grid_constant__ WalkParams a, const __grid_constant__ SobolBase base,
                               uint32_t R, uint32_t r0, uint32_t bits, uint32_t nlev, uint32_t *__restrict__ tabs) {
    const uint32_t id = blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= R * (uint32_t)QMC_DIMS) return;
    const uint32_t r = r0 + id / QMC_DIMS, d = id % QMC_DIMS;  // r: the replicate's global index
    uint32_t row[32];
#pragma unroll
    for (uint32_t b = 0; b < 32; ++b) {
        const uint32_t above = b == 0 ? 0u : (0xFFFFFFFFu << (32u - b));
        row[b] = (philox_rk(make_uint4(b, STREAM_SCRAMBLE, d, r), a).x & above) | (0x80000000u >> b);
    }
    uint32_t *out = tabs + (uint64_t)id * nlev * 32u;
    for (uint32_t l = 0; l < nlev; ++l) {
        uint32_t v[QMC_DIGIT];
#pragma unroll
        for (uint32_t j = 0; j < QMC_DIGIT; ++j) {
            const uint32_t b = l * QMC_DIGIT + j;
            uint32_t y = 0;
            if (b < bits) {
                const uint32_t x = base.v[d][b];
#pragma unroll
                for (uint32_t k = 0; k < 32; ++k) y |= ((uint32_t)__popc(row[k] & x) & 1u) << (31u - k);
            }
            v[j] = y;
        }
        for (uint32_t c = 0; c < 32; ++c) {
            uint32_t x = 0;
#pragma unroll
            for (uint32_t j = 0; j < QMC_DIGIT; ++j)
                if ((c >> j) & 1u) x ^= v[j];
            out[l * 32u + c] = x;
        }
    }
}

// Coordinate of point q from one dimension's digit tables.
__device__ __forceinline__ uint32_t sobol_coord(const uint32_t *__restrict__ tab, uint32_t q, uint32_t nlev) {
    uint32_t x = 0;
#pragma unroll
    for (uint32_t l = 0; l < QMC_LEVELS; ++l)
        if (l < nlev) x ^= __ldg(tab + l * 32u + ((q >> (l * QMC_DIGIT)) & 31u));
    return x;
}

struct RqmcJob {
    uint32_t log2q;        // points per replicate: 2^log2q
    uint32_t R;            // replicates
    uint32_t r0;           // global index of replicate 0 (scrambles, shifts, path indices)
    uint32_t G;            // replicates per warp (slices == 1)
    uint32_t groups;       // ceil(R / G)
    uint32_t slices;       // warps per replicate (a power of two <= 2^log2q; G == 1 when > 1)
    bool fused;            // G == R and slices == 1: each warp finishes its entry's statistics
    uint32_t nlev;         // digit levels: ceil(log2q / 5)
    const uint32_t *tabs;  // [R][QMC_DIMS][nlev][32] digit tables of the scrambled points
    double2 *part;         // [n_entries][R][slices]: {sum of e^{logW - m} v, m}
};

// Per-warp shared buffer: the digital shifts of the replicates in flight (one
// at a time for replicates of 32 points or more, else 32 / 2^log2q at a time).
constexpr int QMC_WARP_WORDS = 32 * QMC_DIMS;

// Shifts e_(i,r,d) of replicates r0 .. r0+nrep-1 into sh[(r - r0) * QMC_DIMS + d]:
// word d mod 4 of Philox {d / 4, 0xFFFFFFFD, i, r}, one block per lane and round.
__device__ __forceinline__ void load_shifts(uint32_t *sh, const WalkParams &a, int32_t i, uint32_t r0, uint32_t nrep,
                                            int lane) {
    for (uint32_t b = (uint32_t)lane; b < nrep * (QMC_DIMS / 4); b += 32) {
        const uint32_t rr = b / (QMC_DIMS / 4), j = b % (QMC_DIMS / 4);
        const uint4 w = philox_rk(make_uint4(j, STREAM_SHIFT, (uint32_t)i, r0 + rr), a);
        uint32_t *o = sh + rr * QMC_DIMS + 4 * j;
        o[0] = w.x;
        o[1] = w.y;
        o[2] = w.z;
        o[3] = w.w;
    }
}

// The event's draw: Philox block of the path, words 0 and 2 replaced by the
// scrambled, shifted Sobol' coordinates for the first QMC_EVENTS events.
__device__ __forceinline__ uint4 qmc_draw(const WalkParams &a, uint32_t k, int32_t i, uint64_t path, uint32_t q,
                                          const uint32_t *tab, uint32_t nlev, const uint32_t *sh) {
    uint4 rnd = philox_rk(make_uint4(k, (uint32_t)i, (uint32_t)path, (uint32_t)(path >> 32)), a);
    if (k < QMC_EVENTS) {
        rnd.x = sobol_coord(tab + (2u * k) * nlev * 32u, q, nlev) ^ sh[2u * k];
        rnd.z = sobol_coord(tab + (2u * k + 1u) * nlev * 32u, q, nlev) ^ sh[2u * k + 1u];
    }
    return rnd;
}

// Replicate-level statistics of one warp: the replicate means
// y_r = S_r e^{m_r - mref} / 2^m kept as differences from the first one (a
// pivot, so that the small spread of the y_r does not cancel), with a
// compensated sum; a replicate with a much larger shift rescales the state.
template <typename T>
struct RepAcc {
    T mref = 0, y0 = 0, sd = 0, cd = 0, sd2 = 0;
    uint32_t n = 0;
    static __device__ __forceinline__ T ex(T x) {
        if constexpr (std::is_same<T, float>::value) return expf(x);
        else return exp(x);
    }
    __device__ __forceinline__ void add(T m, T y) {  // y: replicate sum / 2^m at shift m
        if (n == 0) {
            mref = m;
            y0 = y;
            n = 1;
            return;
        }
        if (!(m <= mref + (T)8)) {  // a larger shift (or a non-finite one): rescale
            const T sc = ex(mref - m);
            y0 *= sc; sd *= sc; cd *= sc; sd2 *= sc * sc;
            mref = m;
        }
        const T d = y * ex(m - mref) - y0;
        const T yk = d - cd;  // compensated sum of the differences
        const T tk = sd + yk;
        cd = (tk - sd) - yk;
        sd = tk;
        sd2 += d * d;
        ++n;
    }
};

// Sum of the lanes' shifted weights and the common shift (FP32 lanes).
__device__ __forceinline__ void merge_lanes(const Acc32 &acc, float &sum, float &mw) {
    mw = acc.m;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mw = fmaxf(mw, __shfl_xor_sync(0xffffffffu, mw, o));
    const float sc = (acc.m == -INFINITY) ? 0.0f : expf(__fsub_rn(acc.m, mw));
    float h = __fmul_rn(acc.s1, sc), l = __fmul_rn(-acc.c1, sc);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        pair_add(h, l, __shfl_xor_sync(0xffffffffu, h, o), __shfl_xor_sync(0xffffffffu, l, o));
    sum = __fadd_rn(h, l);
}
__device__ __forceinline__ void merge_lanes(const Acc64 &acc, double &sum, double &mw) {
    double s2;
    acc.warp_merge(sum, s2, mw);
}

// Segmented merge over aligned groups of `width` lanes (a power of two <= 32):
// the group's shift and its sum of e^{L - shift} v.
__device__ __forceinline__ void merge_segment(float L, float v, bool valid, uint32_t width, float &sum, float &mx) {
    mx = valid ? L : -INFINITY;
    for (uint32_t o = width >> 1; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, (int)o));
    float h = valid ? __fmul_rn(expf(__fsub_rn(L, mx)), v) : 0.0f, l = 0.0f;
    for (uint32_t o = width >> 1; o > 0; o >>= 1)
        pair_add(h, l, __shfl_xor_sync(0xffffffffu, h, (int)o), __shfl_xor_sync(0xffffffffu, l, (int)o));
    sum = __fadd_rn(h, l);
}
__device__ __forceinline__ void merge_segment(double L, double v, bool valid, uint32_t width, double &sum,
                                              double &mx) {
    mx = valid ? L : -INFINITY;
    for (uint32_t o = width >> 1; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, (int)o));
    sum = valid ? exp(L - mx) * v : 0.0;
    for (uint32_t o = width >> 1; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, (int)o);
}

// One warp per (entry, group of G replicates, slice).  The entry row is staged
// once; replicates of >= 32 points run one after another with lane refill over
// their points, smaller ones 32 / 2^log2q at a time with one point per lane and
// a segmented merge over each replicate's lanes.  When a warp holds all
// replicates of its entry (job.fused), it folds the replicate means itself
// (RepAcc) and the last warp of the block finishes the block's entries (mean,
// standard error), one lane per entry; otherwise it writes one partial per
// (replicate, slice) for k_rqmc_finish.
#ifndef MCX_RQMC_MIN_BLOCKS
#define MCX_RQMC_MIN_BLOCKS 4
#endif
template <int MODE, bool WEIGHTED, bool F64, bool SMALLQ>
__global__ void __launch_bounds__(WALK_THREADS, F64 ? WALK_MIN_BLOCKS_F64 : MCX_RQMC_MIN_BLOCKS)
    k_walk_rqmc(const __grid_constant__ WalkParams a, const RqmcJob job) {
    using Q = P<F64>;
    using T = typename Q::T;
    using Acc = typename std::conditional<F64, Acc64, Acc32>::type;
    __shared__ StageWarp s_stage[WARPS_PER_BLOCK];
    __shared__ uint32_t s_buf[WARPS_PER_BLOCK][QMC_WARP_WORDS];
    __shared__ double s_fin[WARPS_PER_BLOCK][5];
    __shared__ unsigned int s_done;
    if (threadIdx.x == 0) s_done = 0u;
    __syncthreads();  // before any warp can arrive at the finish ticket
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const uint64_t wid = (uint64_t)blockIdx.x * WARPS_PER_BLOCK + warp;
    const uint64_t per_entry = (uint64_t)job.groups * job.slices;
    const uint64_t n_jobs = (uint64_t)a.n_entries * per_entry;
    const bool valid = wid < n_jobs;  // warp-uniform
    uint64_t e_idx = 0;
    uint32_t r_begin = 0, r_end = 0, sl = 0;
    int32_t i = 0;
    bool bad = false;
    if (valid) {
        e_idx = wid / per_entry;
        const uint32_t gs = (uint32_t)(wid - e_idx * per_entry);
        const uint32_t g = gs / job.slices;
        sl = gs - g * job.slices;
        r_begin = g * job.G;
        r_end = min(job.R, r_begin + job.G);
        i = a.entries ? __ldg(a.entries + e_idx) : (int32_t)e_idx;
        bad = i < 0 || (int64_t)i >= a.n;  // invalid entry: flagged, NaN results, nothing read
    }
    double2 *out = job.fused ? nullptr : job.part + (e_idx * job.R) * job.slices;  // this entry's partials
    RepAcc<T> rep;
    unsigned long long jumps = 0, paths = 0;
    if (valid && !bad) {
        StageWarp &sw = s_stage[warp];
        const NodeRec start = load_node(a.node, i);
        const bool staged = !F64 && start.deg <= STAGE;
        if (lane == 0) sw.start = start;
        if (staged) stage_row<WEIGHTED>(sw, a, start, lane);
        const StageWarp *swp = staged ? &sw : nullptr;
        const T delta_start = Q::pot(start, a.node64, i);
        const T t0 = F64 ? (T)a.t64 : (T)a.t32;
        const uint32_t bits = job.log2q;
        const uint32_t nlev = job.nlev;
        const uint64_t tab_words = (uint64_t)QMC_DIMS * nlev * 32u;  // digit-table words per replicate
        const T invQ = (T)1 / (T)(1u << bits);  // exact: a power of two
        uint32_t *buf = s_buf[warp];
        Walker<F64> w;

        if (!SMALLQ) {
            // ---- one replicate at a time, lane refill over the slice's points ----
            const uint32_t len = (1u << bits) / job.slices;
            const uint32_t q0 = sl * len;
            uint32_t *sh = buf;
            const unsigned lt_mask = (1u << lane) - 1u;
            for (uint32_t r = r_begin; r < r_end; ++r) {
                __syncwarp();  // the previous replicate's shifts are no longer read
                load_shifts(sh, a, i, job.r0 + r, 1, lane);
                __syncwarp();
                const uint32_t *tab = job.tabs + (uint64_t)r * tab_words;
                const uint64_t pbase = ((uint64_t)(job.r0 + r) << bits) + q0;
                w.rec = sw.start; w.j = i; w.r = t0; w.acc = (T)0; w.delta = delta_start; w.k = 0;
                uint32_t next = 32;  // warp-uniform
                uint32_t p = (uint32_t)lane;
                bool active = p < len;
                Acc acc;
                while (__any_sync(0xffffffffu, active)) {
                    bool fin = false;
                    if (active) {
                        const uint4 rnd = qmc_draw(a, w.k, i, pbase + p, q0 + p, tab, nlev, sh);
                        if (advance_drawn<MODE, WEIGHTED, F64>(w, a, rnd, swp, i)) {
                            fin = true;
                            const T L = final_logw<MODE, F64>(w, delta_start, a);
                            if (F64) acc.add(L, __ldg(&a.node64[w.j].v));
                            else acc.add(L, w.rec.v);
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
                        }
                        next += (uint32_t)__popc(fm);
                    }
                }
                T sum, mw;
                merge_lanes(acc, sum, mw);  // uniform across the warp
                if (job.fused) rep.add(mw, sum * invQ);
                else if (lane == 0) out[r * job.slices + sl] = make_double2((double)sum, (double)mw);
                paths += len;
            }
        } else {
            // ---- 32 / 2^bits replicates per pass, one point per lane ----
            const uint32_t Qn = 1u << bits;
            const uint32_t per = 32u >> bits;
            const uint32_t rl = (uint32_t)lane >> bits, q = (uint32_t)lane & (Qn - 1u);
            uint32_t *sh_all = buf;
            for (uint32_t rb = r_begin; rb < r_end; rb += per) {
                const uint32_t np = min(per, r_end - rb);
                __syncwarp();
                load_shifts(sh_all, a, i, job.r0 + rb, np, lane);
                __syncwarp();
                const bool mine = rl < np;
                T L = (T)0, vend = (T)0;
                if (mine) {
                    const uint64_t path = ((uint64_t)(job.r0 + rb + rl) << bits) + q;
                    w.rec = sw.start; w.j = i; w.r = t0; w.acc = (T)0; w.delta = delta_start; w.k = 0;
                    const uint32_t *tab = job.tabs + (uint64_t)(rb + rl) * tab_words;
                    while (!advance_drawn<MODE, WEIGHTED, F64>(
                        w, a, qmc_draw(a, w.k, i, path, q, tab, nlev, sh_all + rl * QMC_DIMS), swp, i)) {
                    }
                    L = final_logw<MODE, F64>(w, delta_start, a);
                    vend = F64 ? (T)__ldg(&a.node64[w.j].v) : (T)w.rec.v;
                    jumps += w.k;
                }
                T sum, mx;
                merge_segment(L, vend, mine, Qn, sum, mx);
                for (uint32_t rr = 0; rr < np; ++rr) {
                    const T s_r = __shfl_sync(0xffffffffu, sum, (int)(rr << bits));
                    const T m_r = __shfl_sync(0xffffffffu, mx, (int)(rr << bits));
                    if (job.fused) rep.add(m_r, s_r * invQ);
                    else if (lane == 0) out[(rb + rr) * job.slices] = make_double2((double)s_r, (double)m_r);
                }
                paths += (uint64_t)np * Qn;
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) jumps += __shfl_xor_sync(0xffffffffu, jumps, o);
    if (valid && lane == 0) {
        if (bad) atomicOr(a.status, ST_BAD_ENTRY);
        if (paths) {
            unsigned long long *ctr = reinterpret_cast<unsigned long long *>(a.status + 2);
            atomicAdd(ctr, paths);
            atomicAdd(ctr + 1, jumps);
        }
        if (bad && !job.fused)
            for (uint32_t r = r_begin; r < r_end; ++r) out[r * job.slices + sl] = make_double2(QNAN, QNAN);
    }
    if (!job.fused) return;  // uniform across the block
    // each warp leaves its entry's replicate statistics in shared memory; the last
    // warp of the block to arrive finishes all of them, one lane per entry
    unsigned int ticket = 0;
    if (lane == 0) {
        s_fin[warp][0] = (valid && !bad) ? (double)rep.mref : QNAN;
        s_fin[warp][1] = (double)rep.y0;
        s_fin[warp][2] = (double)rep.sd - (double)rep.cd;
        s_fin[warp][3] = (double)rep.sd2;
        s_fin[warp][4] = (double)rep.n;
        __threadfence_block();
        ticket = atomicAdd(&s_done, 1u);
    }
    ticket = __shfl_sync(0xffffffffu, ticket, 0);
    if (ticket == WARPS_PER_BLOCK - 1) {
        __threadfence_block();
        const uint64_t e = (uint64_t)blockIdx.x * WARPS_PER_BLOCK + lane;  // fused: one job per entry
        if (lane < WARPS_PER_BLOCK && e < n_jobs) {
            const volatile double *f = s_fin[lane];
            const double mref = f[0];
            if (isnan(mref)) {
                a.mean[e] = QNAN;
                if (a.sem) a.sem[e] = QNAN;
            } else {
                const double R = f[4], sd = f[2];
                const double scale = exp(mref) * (F64 ? 1.0 : v_scale(a.status));
                const double mv = scale * (f[1] + sd / R);
                double var = R > 1.0 ? (f[3] - sd * sd / R) / (R - 1.0) : 0.0;
                if (var < 0.0) var = 0.0;
                const double se = scale * sqrt(var / R);
                a.mean[e] = mv;
                if (a.sem) a.sem[e] = se;
                if (!isfinite(mv) || !isfinite(se)) atomicOr(a.status, ST_OVERFLOW);
            }
        }
    }
}

// Replicate r of an entry: merge its slices into (sum, shift).
__device__ __forceinline__ void replicate_sum(const double2 *pp, uint32_t slices, double &s, double &m) {
    m = -INFINITY;
    for (uint32_t k = 0; k < slices; ++k) m = fmax(m, pp[k].y);
    s = 0.0;
    for (uint32_t k = 0; k < slices; ++k)
        if (pp[k].y != -INFINITY) s += exp(pp[k].y - m) * pp[k].x;  // NaN or infinite sums propagate
}

// One warp per entry: replicate means mu_r = e^{m_r} s_r / 2^m, then the mean of
// the mu_r and its standard error sqrt(sum (mu_r - mean)^2 / ((R - 1) R)).
// Invalid entries (flagged by the walker) get NaN; any other non-finite result
// sets the overflow flag.
__global__ void __launch_bounds__(WALK_THREADS) k_rqmc_finish(const double2 *__restrict__ part,
                                                             const int32_t *__restrict__ entries, int64_t n,
                                                             int64_t n_entries, uint32_t R, uint32_t slices, double Qn,
                                                             bool v_scaled, double *mean, double *sem,
                                                             uint32_t *status) {
    const int lane = threadIdx.x & 31;
    const int64_t e = ((int64_t)blockIdx.x * WALK_THREADS + threadIdx.x) >> 5;
    if (e >= n_entries) return;
    const int32_t i = entries ? __ldg(entries + e) : (int32_t)e;
    if (i < 0 || (int64_t)i >= n) {
        if (lane == 0) {
            mean[e] = QNAN;
            if (sem) sem[e] = QNAN;
        }
        return;
    }
    const double2 *pe = part + (uint64_t)e * R * slices;
    double M = -INFINITY;
    for (uint32_t r = lane; r < R; r += 32) {
        double s, m;
        replicate_sum(pe + (uint64_t)r * slices, slices, s, m);
        M = fmax(M, m);
    }
    M = warp_max(M);
    double sum = 0.0;
    for (uint32_t r = lane; r < R; r += 32) {
        double s, m;
        replicate_sum(pe + (uint64_t)r * slices, slices, s, m);
        if (m != -INFINITY) sum += exp(m - M) * s / Qn;
    }
    const double mu = warp_sum(sum) / (double)R;
    double ss = 0.0;
    for (uint32_t r = lane; r < R; r += 32) {
        double s, m;
        replicate_sum(pe + (uint64_t)r * slices, slices, s, m);
        const double y = m == -INFINITY ? 0.0 : exp(m - M) * s / Qn;
        ss += (y - mu) * (y - mu);
    }
    ss = warp_sum(ss);
    if (lane == 0) {
        const double scale = (M == -INFINITY ? 0.0 : exp(M)) * (v_scaled ? v_scale(status) : 1.0);
        const double mv = scale * mu;
        const double se = R > 1 ? scale * sqrt(ss / (double)(R - 1) / (double)R) : 0.0;
        mean[e] = mv;
        if (sem) sem[e] = se;
        if (!isfinite(mv) || !isfinite(se)) atomicOr(status, ST_OVERFLOW);
    }
}

template <bool F64, bool WEIGHTED, bool SMALLQ>
cudaError_t launch_rqmc_mode(int mode, unsigned grid, const WalkParams &p, const RqmcJob &j, cudaStream_t st) {
    switch (mode) {
        case MCX_EXACT: k_walk_rqmc<MCX_EXACT, WEIGHTED, F64, SMALLQ><<<grid, WALK_THREADS, 0, st>>>(p, j); break;
        case MCX_STRANG: k_walk_rqmc<MCX_STRANG, WEIGHTED, F64, SMALLQ><<<grid, WALK_THREADS, 0, st>>>(p, j); break;
        default: k_walk_rqmc<MCX_LIE, WEIGHTED, F64, SMALLQ><<<grid, WALK_THREADS, 0, st>>>(p, j); break;
    }
    return cudaGetLastError();
}

template <bool F64, bool WEIGHTED>
cudaError_t launch_rqmc_size(int mode, unsigned grid, const WalkParams &p, const RqmcJob &j, cudaStream_t st) {
    // replicates of fewer than 32 points: several per pass, one point per lane
    return j.log2q < 5 ? launch_rqmc_mode<F64, WEIGHTED, true>(mode, grid, p, j, st)
                       : launch_rqmc_mode<F64, WEIGHTED, false>(mode, grid, p, j, st);
}

}  // namespace

cudaError_t launch_estimate_rqmc(mcx_plan *plan, const RqmcArgs &a, cudaStream_t st) {
    if (a.n_entries == 0) return cudaSuccess;
    WalkParams p = make_params(plan, a.t, a.mode == MCX_EXACT ? 1 : a.nsteps, a.seed);
    p.entries = a.entries;
    p.n_entries = a.n_entries;
    p.mean = a.mean;
    p.sem = a.sem;
    const uint32_t Qn = 1u << a.log2q;
    // slices: cut replicates while the GPU would otherwise hold fewer than ~8
    // waves of warps, keeping at least 1024 points per warp
    // Many entries: a warp takes G replicates of one entry (its row staged once),
    // G as large as keeps ~8 waves of warps.  Few entries: one replicate per warp,
    // cut into slices of at least 1024 points while the GPU would hold fewer warps.
    const uint64_t target_warps = 152ull * 64ull * 8ull;
    const uint64_t units = (uint64_t)a.n_entries * a.replicates;
    uint32_t slices = 1, G = 1;
    if (units >= target_warps) {
        const uint64_t gg = units / target_warps;
        G = (uint32_t)(gg < a.replicates ? gg : a.replicates);
    } else {
        while (units * slices < target_warps && Qn / slices >= 2048u) slices *= 2;
    }
    const uint32_t groups = (a.replicates + G - 1) / G;
    const uint64_t jobs = (uint64_t)a.n_entries * groups * slices;
    const uint64_t grid64 = (jobs + WARPS_PER_BLOCK - 1) / WARPS_PER_BLOCK;
    if (grid64 > 0x7FFFFFFFull) return cudaErrorInvalidValue;
    RqmcJob job{};
    job.log2q = a.log2q;
    job.R = a.replicates;
    job.r0 = a.r0;
    job.G = G;
    job.groups = groups;
    job.slices = slices;
    job.fused = groups == 1 && slices == 1;
    const uint32_t nlev = (a.log2q + QMC_DIGIT - 1) / QMC_DIGIT;
    job.nlev = nlev;
    void *tabs = nullptr, *part = nullptr;
    const size_t tab_bytes = sizeof(uint32_t) * (size_t)a.replicates * QMC_DIMS * nlev * 32u;
    cudaError_t e = cudaSuccess;
    if (tab_bytes > 0) e = pool_alloc(&tabs, tab_bytes, st);
    if (e == cudaSuccess && !job.fused) e = pool_alloc(&part, sizeof(double2) * (size_t)(units * slices), st);
    if (e == cudaSuccess && tab_bytes > 0) {
        const uint32_t threads = a.replicates * (uint32_t)QMC_DIMS;
        k_qmc_scramble<<<(threads + 127) / 128, 128, 0, st>>>(p, sobol_base(), a.replicates, a.r0, a.log2q, nlev,
                                                              static_cast<uint32_t *>(tabs));
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        job.tabs = static_cast<const uint32_t *>(tabs);
        job.part = static_cast<double2 *>(part);
        const bool weighted = plan->weighted_rows > 0;
        const unsigned grid = (unsigned)grid64;
        if (a.precision == MCX_FP64)
            e = weighted ? launch_rqmc_size<true, true>(a.mode, grid, p, job, st)
                         : launch_rqmc_size<true, false>(a.mode, grid, p, job, st);
        else
            e = weighted ? launch_rqmc_size<false, true>(a.mode, grid, p, job, st)
                         : launch_rqmc_size<false, false>(a.mode, grid, p, job, st);
    }
    if (e == cudaSuccess && !job.fused) {
        const unsigned g2 = (unsigned)((a.n_entries + WARPS_PER_BLOCK - 1) / WARPS_PER_BLOCK);
        k_rqmc_finish<<<g2, WALK_THREADS, 0, st>>>(job.part, a.entries, plan->n, a.n_entries, a.replicates, slices,
                                                   (double)Qn, a.precision != MCX_FP64, a.mean, a.sem, plan->status);
        e = cudaGetLastError();
    }
    if (tabs) pool_free(tabs, st);
    if (part) pool_free(part, st);
    return e;
}

}  // namespace mcx
