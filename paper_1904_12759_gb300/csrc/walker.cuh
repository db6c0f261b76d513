// Walker core shared by the estimate, forward, quasi-random and batch
// kernels: launch parameters (and their construction from a plan),
// Philox4x32-10 with precomputed round keys, the staging of an entry row in
// shared memory, the FP32/FP64 precision traits and the one-event step
// `advance` / `advance_drawn` (Sec. 3, Eq. paths: exponential holding time,
// stop at the horizon, jump by the row's table), plus the final log-weight of
// each functional (Theorem 1; Eqs. deff and eq_general1).  See walk.cu for the
// path arithmetic.
#pragma once

#include <math.h>

#include "mcx_internal.cuh"

namespace mcx {
namespace {

constexpr int WALK_THREADS = 256;
constexpr int WARPS_PER_BLOCK = WALK_THREADS / 32;
constexpr int STAGE = 32;  // max staged entry-row length
constexpr uint64_t LANE_MODE_MAX_PATHS = 64;  // at most this many paths per entry: one lane per entry
#ifndef MCX_WALK_MIN_BLOCKS
#define MCX_WALK_MIN_BLOCKS 6
#endif
// resident blocks per SM requested from the compiler: FP32 walkers 6 (48 warps,
// <= 42 registers); the FP64 path version keeps more registers
constexpr int WALK_MIN_BLOCKS_F32 = MCX_WALK_MIN_BLOCKS;
constexpr int WALK_MIN_BLOCKS_F64 = 4;
constexpr uint64_t FNV_OFFSET = 14695981039346656037ull;
constexpr uint64_t FNV_PRIME = 1099511628211ull;
constexpr double QNAN = __builtin_nan("");

struct Partial {
    double s1;  // sum of e^{logW - m} v
    double s2;  // sum of (e^{logW - m} v)^2
    double m;   // shift
};

struct WalkParams {
    const NodeRec *node;
    const NodeRec64 *node64;
    const int32_t *edge_col;
    const Edge16 *edge16;  // weighted plans: packed column + alias records
    const int32_t *entries;
    int64_t n_entries;
    uint64_t paths;       // per entry
    uint64_t chunk_len;   // paths per warp
    uint32_t chunks_per_entry;
    int nsteps;
    int64_t n;            // rows: entries outside [0, n) are rejected
    uint32_t max_events;  // per-path event cap (guarantees termination)
    double t64, dt64, invdt64;
    float t32, dt32, invdt32;
    uint32_t rk0[10], rk1[10];  // Philox round keys: seed + r * (Weyl increments)
    uint64_t path_offset;
    double *mean;
    double *sem;
    Partial *partials;    // [n_entries * chunks_per_entry] when chunks_per_entry > 1
    uint32_t *status;
};

// The entry row of one warp, staged in shared memory.
struct StageWarp {
    NodeRec start;               // the entry's own record
    NodeRec rec[STAGE];          // records of its kept columns
    int32_t col[STAGE];          // kept columns (CSR order)
    int32_t aslot[STAGE];        // alias rows: slot of the alias column
    uint32_t thresh[STAGE];      // alias rows: keep-own-column threshold
};

// Round keys of Philox4x32-10 for key = seed: the key words bumped by the
// Weyl constants before each round.
inline void set_round_keys(WalkParams &p, uint64_t seed) {
    uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    for (int r = 0; r < 10; ++r) {
        p.rk0[r] = k0;
        p.rk1[r] = k1;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

// Walk parameters of a plan for horizon t, N grid steps and the given seed.
inline WalkParams make_params(mcx_plan *plan, double t, int nsteps, uint64_t seed) {
    WalkParams p{};
    p.node = plan->node;
    p.node64 = plan->node64;
    p.edge_col = plan->edge_col;
    p.edge16 = plan->edge16;
    p.nsteps = nsteps;
    p.t64 = t;
    p.dt64 = t / (double)nsteps;
    p.invdt64 = (double)nsteps / t;
    p.t32 = (float)t;
    p.dt32 = (float)p.dt64;
    p.invdt32 = (float)p.invdt64;
    p.n = plan->n;
    p.max_events = 1u << 30;
    set_round_keys(p, seed);
    p.status = plan->status;
    return p;
}

// Stage the row of an entry with record `start` (deg <= STAGE) into sw: its
// kept columns, their node records and, for weighted rows, the alias slots and
// thresholds.  Called by the whole warp; sw.start is set by the caller.
template <bool WEIGHTED>
__device__ __forceinline__ void stage_row(StageWarp &sw, const WalkParams &a, const NodeRec &start, int lane) {
    for (int k = lane; k < start.deg; k += 32) {
        const int32_t c = __ldg(a.edge_col + start.row_start + k);
        sw.col[k] = c;
        sw.rec[k] = load_node(a.node, c);
    }
    __syncwarp();
    if (WEIGHTED && (start.flags & NODE_WEIGHTED)) {
        for (int k = lane; k < start.deg; k += 32) {
            const Edge16 ed = a.edge16[start.row_start + k];
            int32_t s2 = k;
            for (int q = 0; q < start.deg; ++q)
                if (sw.col[q] == ed.alias_col) s2 = q;
            sw.aslot[k] = s2;
            sw.thresh[k] = ed.thresh;
        }
    }
}

// Philox4x32-10 with the ten round keys precomputed on the host.
__device__ __forceinline__ uint4 philox_rk(uint4 c, const WalkParams &a) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x;
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ a.rk0[r], lo1, hi0 ^ c.w ^ a.rk1[r], lo0);
    }
    return c;
}

// ---------------------------------------------------------------------------
// Precision traits: the same path code in FP32 and FP64.
// ---------------------------------------------------------------------------
template <bool F64>
struct P;

template <>
struct P<false> {
    using T = float;
    static __device__ __forceinline__ T unif(uint4 w) { return unif24(w.x); }
    static __device__ __forceinline__ T neg_ln(T u) { return -ln_f32(u); }
    static __device__ __forceinline__ T mul(T a, T b) { return __fmul_rn(a, b); }
    static __device__ __forceinline__ T sub(T a, T b) { return __fsub_rn(a, b); }
    static __device__ __forceinline__ T fma(T a, T b, T c) { return __fmaf_rn(a, b, c); }
    static __device__ __forceinline__ T from_int(int c) { return __int2float_rn(c); }
    static __device__ __forceinline__ int grid(T rho, T invdt, int N) {
        if (rho < 0.0f) return 0;
        const T f = floorf(__fmul_rn(rho, invdt));
        const int c = (int)f + 1;
        return c < N ? c : N;
    }
    static __device__ __forceinline__ T rate(const NodeRec &r, const NodeRec64 *, int32_t) { return r.inv_rate; }
    static __device__ __forceinline__ T pot(const NodeRec &r, const NodeRec64 *, int32_t) { return r.delta; }
};

template <>
struct P<true> {
    using T = double;
    static __device__ __forceinline__ T unif(uint4 w) { return unif53(w.x, w.y); }
    static __device__ __forceinline__ T neg_ln(T u) { return -ln_f64(u); }
    static __device__ __forceinline__ T mul(T a, T b) { return __dmul_rn(a, b); }
    static __device__ __forceinline__ T sub(T a, T b) { return __dsub_rn(a, b); }
    static __device__ __forceinline__ T fma(T a, T b, T c) { return __fma_rn(a, b, c); }
    static __device__ __forceinline__ T from_int(int c) { return __int2double_rn(c); }
    static __device__ __forceinline__ int grid(T rho, T invdt, int N) {
        if (rho < 0.0) return 0;
        const T f = floor(__dmul_rn(rho, invdt));
        const int c = (int)f + 1;
        return c < N ? c : N;
    }
    static __device__ __forceinline__ T rate(const NodeRec &, const NodeRec64 *n64, int32_t j) {
        return __ldg(&n64[j].inv_rate);
    }
    static __device__ __forceinline__ T pot(const NodeRec &, const NodeRec64 *n64, int32_t j) {
        return __ldg(&n64[j].delta);
    }
};

// One walker between events.
template <bool F64>
struct Walker {
    using T = typename P<F64>::T;
    NodeRec rec;  // record of the current state j
    int32_t j;
    T r;          // remaining time
    T acc;        // EXACT: running logW; grid modes: sum delta * grid count
    T delta;      // potential of the current state
    uint32_t k;   // event counter
};

// Advance one event with the event's draw `rnd` given (word 0: holding-time
// uniform, with word 1 in FP64; word 2: slot; word 3: alias acceptance).
// Returns true when the path has ended (then w.acc holds the final accumulated
// value with the last hold included).  With `sw` set, jumps out of state `i0`
// read the staged row.
template <int MODE, bool WEIGHTED, bool F64>
__device__ __forceinline__ bool advance_drawn(Walker<F64> &w, const WalkParams &a, uint4 rnd, const StageWarp *sw,
                                              int32_t i0, typename P<F64>::T *hold = nullptr) {
    using Q = P<F64>;
    using T = typename Q::T;
    const T invdt = F64 ? (T)a.invdt64 : (T)a.invdt32;
    const int N = a.nsteps;
    // -ln(u) does not depend on the state, so it is computed before the state's
    // record (often still in flight from the last jump) is used; a state without
    // jumps simply ignores it
    const T e = Q::neg_ln(Q::unif(rnd));
    if (w.rec.deg == 0 || w.k >= a.max_events) {
        if (w.rec.deg != 0) atomicOr(a.status, ST_OVERFLOW);  // event cap reached: result flagged
        w.acc = MODE == MCX_EXACT ? Q::fma(w.delta, w.r, w.acc) : Q::fma(w.delta, Q::from_int(Q::grid(w.r, invdt, N)), w.acc);
        if (hold) *hold = w.r;
        return true;
    }
    const T S = Q::mul(e, Q::rate(w.rec, a.node64, w.j));
    if (S >= w.r) {
        w.acc = MODE == MCX_EXACT ? Q::fma(w.delta, w.r, w.acc) : Q::fma(w.delta, Q::from_int(Q::grid(w.r, invdt, N)), w.acc);
        if (hold) *hold = w.r;
        return true;
    }
    if (hold) *hold = S;
    const T rn = Q::sub(w.r, S);
    if (MODE == MCX_EXACT) {
        w.acc = Q::fma(w.delta, S, w.acc);
    } else {
        w.acc = Q::fma(w.delta, Q::from_int(Q::grid(w.r, invdt, N) - Q::grid(rn, invdt, N)), w.acc);
    }
    w.r = rn;
    const uint32_t slot = __umulhi(rnd.z, (uint32_t)w.rec.deg);
    int32_t c;
    if (sw != nullptr && w.j == i0) {
        uint32_t s2 = slot;
        if (WEIGHTED && (w.rec.flags & NODE_WEIGHTED) && !(rnd.w < sw->thresh[slot])) s2 = (uint32_t)sw->aslot[slot];
        c = sw->col[s2];
        w.rec = sw->rec[s2];
    } else {
        const int64_t e = w.rec.row_start + slot;
        if (WEIGHTED) {  // one 16-byte record: own column, alias column, threshold
            const int4 ed = __ldg(reinterpret_cast<const int4 *>(a.edge16 + e));
            c = (rnd.w < (uint32_t)ed.z) ? ed.x : ed.y;
        } else {
            c = __ldg(a.edge_col + e);
        }
        w.rec = load_node(a.node, c);
    }
    w.j = c;
    w.delta = Q::pot(w.rec, a.node64, c);
    ++w.k;
    return false;
}

// Advance one event with the path's own Philox block {k, stream, path}.
template <int MODE, bool WEIGHTED, bool F64>
__device__ __forceinline__ bool advance(Walker<F64> &w, const WalkParams &a, uint32_t stream, uint64_t path,
                                        const StageWarp *sw, int32_t i0,
                                        typename P<F64>::T *hold = nullptr) {
    const uint4 rnd = philox_rk(make_uint4(w.k, stream, (uint32_t)path, (uint32_t)(path >> 32)), a);
    return advance_drawn<MODE, WEIGHTED, F64>(w, a, rnd, sw, i0, hold);
}

template <int MODE, bool F64>
__device__ __forceinline__ typename P<F64>::T final_logw(const Walker<F64> &w, typename P<F64>::T delta_start,
                                                         const WalkParams &a) {
    using Q = P<F64>;
    using T = typename Q::T;
    const T dt = F64 ? (T)a.dt64 : (T)a.dt32;
    if (MODE == MCX_EXACT) return w.acc;
    if (MODE == MCX_LIE) return Q::mul(w.acc, dt);
    T s = Q::fma((T)0.5, delta_start, w.acc);
    s = Q::fma((T)-0.5, w.delta, s);
    return Q::mul(s, dt);
}

}  // namespace
}  // namespace mcx
