// Backward walkers (Theorem 1, Algorithm 1) and the segmented per-entry
// reduction.
//
// Work decomposition: the paths of each requested entry are split into
// chunks of `chunk_len` consecutive path indices; one warp owns one
// (entry, chunk).  Each lane runs paths p = chunk_begin + lane, +32, ... one
// after another in a single flat event loop: every iteration draws one
// Philox block and either finishes the lane's current path (folding its
// weight into the lane's accumulators and starting the next path from the
// entry) or takes one jump.  A lane whose path ends takes the next unassigned
// path of the chunk, so the lanes stay busy until the chunk is exhausted.  A jump is two dependent random
// gathers: the column (4 B) and the new node's 32-byte record.
//
// Hot-row staging: every path of a warp starts at the same entry, so the
// entry's row (its kept columns, their node records and alias slots, up to
// STAGE entries) is staged in shared memory once per warp; jumps out of the
// entry state read shared memory instead of two dependent global gathers.
//
// Path arithmetic (every op a single IEEE operation or an explicit fma):
//   S = (-ln u) * inv_rate_j          holding time in state j
//   S >= r  -> stop;  else r <- r - S, jump
//   EXACT : logW += delta_j * hold         (hold = S, or r for the last hold)
//   grid  : acc  += delta_j * (#grid points m*dt, m = 0..N-1, inside the hold,
//                              counted in remaining time); LIE logW = acc*dt;
//           STRANG logW = (acc + delta_start/2 - delta_end/2)*dt
// Weights: FP32 paths accumulate w = e^{logW - m} v (m a per-lane running
// shift) with compensated FP32 sums of w and w^2; lanes merge with
// compensated FP32 pairs after log-sum-exp rescaling, so the FP64 pipe (slow
// on this GPU) is used only per warp and per entry; each block then finishes
// its entries (mean, standard error) with one lane per entry.  Entries split
// into several chunks merge their chunk partials in FP64 in chunk order
// (k_reduce_chunks).  FP64 paths do all of this in FP64.
#include <math.h>

#include <mutex>
#include <type_traits>

#include "accum.cuh"
#include "launch.h"
#include "walker.cuh"

namespace mcx {
namespace {

// ---------------------------------------------------------------------------
// Estimate kernel: one warp per (entry, chunk); a block finishes its entries.
// ---------------------------------------------------------------------------
template <int MODE, bool WEIGHTED, bool F64>
__global__ void __launch_bounds__(WALK_THREADS, F64 ? WALK_MIN_BLOCKS_F64 : WALK_MIN_BLOCKS_F32)
    k_walk(const __grid_constant__ WalkParams a) {
    using Q = P<F64>;
    using T = typename Q::T;
    using Acc = typename std::conditional<F64, Acc64, Acc32>::type;
    __shared__ StageWarp s_stage[WARPS_PER_BLOCK];
    __shared__ double s_fin[WARPS_PER_BLOCK][3];
    __shared__ unsigned int s_done;
    if (threadIdx.x == 0) s_done = 0u;
    __syncthreads();  // before any warp can arrive at the finish ticket
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const uint64_t wid = (uint64_t)blockIdx.x * WARPS_PER_BLOCK + warp;
    const uint64_t n_chunks = (uint64_t)a.n_entries * a.chunks_per_entry;
    const bool valid = wid < n_chunks;  // uniform across the warp
    uint64_t e_idx = 0, chunk = 0;
    int32_t i = 0;
    bool bad = false;
    if (valid) {
        e_idx = wid / a.chunks_per_entry;
        chunk = wid - e_idx * a.chunks_per_entry;
        i = a.entries ? __ldg(a.entries + e_idx) : (int32_t)e_idx;
        bad = i < 0 || (int64_t)i >= a.n;  // invalid entry: flagged, outputs NaN, nothing read
    }
    double S1 = 0.0, S2 = 0.0, Mw = QNAN;
    if (valid && !bad) {
        const uint64_t p_begin = chunk * a.chunk_len;
        const uint64_t p_end = min(a.paths, p_begin + a.chunk_len);
        StageWarp &sw = s_stage[warp];
        const NodeRec start = load_node(a.node, i);
        // stage the entry row (FP32 paths only; the FP64 path version reads global memory)
        const bool staged = !F64 && start.deg <= STAGE;
        if (lane == 0) sw.start = start;  // every path restarts from this copy
        if (staged) stage_row<WEIGHTED>(sw, a, start, lane);
        __syncwarp();
        const StageWarp *swp = staged ? &sw : nullptr;
        const T delta_start = Q::pot(start, a.node64, i);
        const T t0 = F64 ? (T)a.t64 : (T)a.t32;

        Walker<F64> w;
        w.rec = start; w.j = i; w.r = t0; w.acc = (T)0; w.delta = delta_start; w.k = 0;
        // lane refill: a lane whose path ends takes the next unassigned path of the
        // chunk (ranked among the lanes finishing in the same iteration), so all
        // lanes run until the chunk is exhausted and finish within about one path
        const uint64_t base = a.path_offset + p_begin;
        const uint32_t len = (uint32_t)(p_end - p_begin);  // chunks are shorter than 2^31 paths
        uint32_t next = 32;                                // warp-uniform
        uint32_t p = (uint32_t)lane;
        bool active = p < len;
        Acc acc;
        uint32_t jumps = 0;
        const unsigned lt_mask = (1u << lane) - 1u;
        while (__any_sync(0xffffffffu, active)) {
            bool fin = false;
            if (active && advance<MODE, WEIGHTED, F64>(w, a, (uint32_t)i, base + p, swp, i)) {
                fin = true;
                const T L = final_logw<MODE, F64>(w, delta_start, a);
                if (F64) acc.add(L, __ldg(&a.node64[w.j].v));
                else acc.add(L, w.rec.v);
                jumps += w.k;
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
        // walker statistics: paths and jumps of this warp, one atomic per warp
        unsigned long long jl = jumps;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) jl += __shfl_xor_sync(0xffffffffu, jl, o);
        if (lane == 0) {
            unsigned long long *ctr = reinterpret_cast<unsigned long long *>(a.status + 2);
            atomicAdd(ctr, (unsigned long long)(p_end - p_begin));
            atomicAdd(ctr + 1, jl);
        }
        acc.warp_merge(S1, S2, Mw);
    }
    if (a.chunks_per_entry == 1) {
        // each warp leaves its sums in shared memory; the last warp of the block
        // to arrive finishes all of them, one lane per entry (no block barrier)
        unsigned int ticket = 0;
        if (lane == 0) {
            s_fin[warp][0] = S1;
            s_fin[warp][1] = S2;
            s_fin[warp][2] = Mw;
            __threadfence_block();
            ticket = atomicAdd(&s_done, 1u);
        }
        ticket = __shfl_sync(0xffffffffu, ticket, 0);
        if (ticket == WARPS_PER_BLOCK - 1) {
            __threadfence_block();
            const uint64_t e = (uint64_t)blockIdx.x * WARPS_PER_BLOCK + lane;
            if (lane < WARPS_PER_BLOCK && e < n_chunks) {
                const double m = ((volatile double *)s_fin[lane])[2];
                if (isnan(m)) {  // invalid entry
                    atomicOr(a.status, ST_BAD_ENTRY);
                    a.mean[e] = QNAN;
                    if (a.sem) a.sem[e] = QNAN;
                } else {
                    finish_entry(((volatile double *)s_fin[lane])[0], ((volatile double *)s_fin[lane])[1], m,
                                 (double)a.paths, F64 ? 1.0 : v_scale(a.status), a.mean + e,
                                 a.sem ? a.sem + e : nullptr, a.status);
                }
            }
        }
    } else if (valid && lane == 0) {
        if (bad) atomicOr(a.status, ST_BAD_ENTRY);
        a.partials[wid] = Partial{bad ? QNAN : S1, S2, bad ? 0.0 : Mw};
    }
}

// One warp per entry: merge its chunk partials in chunk order (v_scaled: the
// partials come from FP32 paths over the scaled copy of v).
__global__ void __launch_bounds__(WALK_THREADS) k_reduce_chunks(const Partial *__restrict__ part, int64_t n_entries,
                                                               uint32_t cpe, double M, bool v_scaled, double *mean,
                                                               double *sem, uint32_t *status) {
    const int lane = threadIdx.x & 31;
    const int64_t e = ((int64_t)blockIdx.x * WALK_THREADS + threadIdx.x) >> 5;
    if (e >= n_entries) return;
    const Partial *pp = part + (uint64_t)e * cpe;
    double m = -INFINITY;
    for (uint32_t c = lane; c < cpe; c += 32) m = fmax(m, pp[c].m);
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
    if (lane == 0) finish_entry(s1, s2, m, M, v_scaled ? v_scale(status) : 1.0, mean + e, sem ? sem + e : nullptr, status);
}

// ---------------------------------------------------------------------------
// Few paths per entry (M <= LANE_MODE_MAX_PATHS): one lane per entry.  The
// lane runs the entry's paths in path order, keeps its own accumulators and
// writes the entry's mean and standard error; no partials, no scratch.
// ---------------------------------------------------------------------------
template <int MODE, bool WEIGHTED, bool F64>
__global__ void __launch_bounds__(WALK_THREADS) k_walk_lanes(const __grid_constant__ WalkParams a) {
    using Q = P<F64>;
    using T = typename Q::T;
    using Acc = typename std::conditional<F64, Acc64, Acc32>::type;
    const int64_t e = (int64_t)blockIdx.x * WALK_THREADS + threadIdx.x;
    const bool valid = e < a.n_entries;  // lanes past the end stay for the warp reduction below
    unsigned long long jumps = 0, paths = 0;
    if (valid) {
        const int32_t i = a.entries ? __ldg(a.entries + e) : (int32_t)e;
        if (i < 0 || (int64_t)i >= a.n) {
            atomicOr(a.status, ST_BAD_ENTRY);
            a.mean[e] = QNAN;
            if (a.sem) a.sem[e] = QNAN;
        } else {
            const NodeRec start = load_node(a.node, i);
            const T delta_start = Q::pot(start, a.node64, i);
            const T t0 = F64 ? (T)a.t64 : (T)a.t32;
            Acc acc;
            for (uint64_t p = 0; p < a.paths; ++p) {
                Walker<F64> w;
                w.rec = start; w.j = i; w.r = t0; w.acc = (T)0; w.delta = delta_start; w.k = 0;
                while (!advance<MODE, WEIGHTED, F64>(w, a, (uint32_t)i, a.path_offset + p, nullptr, i)) {
                }
                const T L = final_logw<MODE, F64>(w, delta_start, a);
                if (F64) acc.add(L, __ldg(&a.node64[w.j].v));
                else acc.add(L, w.rec.v);
                jumps += w.k;
            }
            paths = a.paths;
            double S1, S2, M;
            acc.lane_result(S1, S2, M);
            finish_entry(S1, S2, M, (double)a.paths, F64 ? 1.0 : v_scale(a.status), a.mean + e,
                         a.sem ? a.sem + e : nullptr, a.status);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        jumps += __shfl_xor_sync(0xffffffffu, jumps, o);
        paths += __shfl_xor_sync(0xffffffffu, paths, o);
    }
    if ((threadIdx.x & 31) == 0 && paths) {
        unsigned long long *ctr = reinterpret_cast<unsigned long long *>(a.status + 2);
        atomicAdd(ctr, paths);
        atomicAdd(ctr + 1, jumps);
    }
}

// ---------------------------------------------------------------------------
// Trace kernel: one thread per path, same stepping code (no staging), plus the
// index hash.
// ---------------------------------------------------------------------------
template <int MODE, bool WEIGHTED, bool F64>
__global__ void __launch_bounds__(WALK_THREADS) k_trace(const __grid_constant__ WalkParams a, int32_t i,
                                                       uint64_t first_path, uint32_t count, int32_t *end,
                                                       uint32_t *njumps, uint64_t *hash, double *logw) {
    using Q = P<F64>;
    using T = typename Q::T;
    const uint32_t q = blockIdx.x * WALK_THREADS + threadIdx.x;
    if (q >= count) return;
    const uint64_t path = first_path + q;
    const NodeRec start = load_node(a.node, i);
    const T delta_start = Q::pot(start, a.node64, i);
    Walker<F64> w;
    w.rec = start; w.j = i; w.r = F64 ? (T)a.t64 : (T)a.t32; w.acc = (T)0; w.delta = delta_start; w.k = 0;
    uint64_t h = (FNV_OFFSET ^ (uint64_t)(uint32_t)i) * FNV_PRIME;
    while (!advance<MODE, WEIGHTED, F64>(w, a, (uint32_t)i, path, nullptr, i))
        h = (h ^ (uint64_t)(uint32_t)w.j) * FNV_PRIME;
    end[q] = w.j;
    njumps[q] = w.k;
    hash[q] = h;
    logw[q] = (double)final_logw<MODE, F64>(w, delta_start, a);
}

__global__ void k_trace_t0(int32_t i, uint32_t count, int32_t *end, uint32_t *njumps, uint64_t *hash, double *logw) {
    const uint32_t q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= count) return;
    end[q] = i;
    njumps[q] = 0;
    hash[q] = (FNV_OFFSET ^ (uint64_t)(uint32_t)i) * FNV_PRIME;
    logw[q] = 0.0;
}

// Exponent of the largest finite |v_i| into status word STATUS_VEXP (biased;
// the word is cleared before the launch).
__global__ void k_v_exponent(int64_t n, const double *__restrict__ v, uint32_t *status) {
    exponent_max(n, v, status + STATUS_VEXP);
}

// v into the node records: FP64 as given, FP32 scaled by 2^-k (exact; see v_scale).
__global__ void k_pack_v(int64_t n, const double *__restrict__ v, NodeRec *__restrict__ node,
                         NodeRec64 *__restrict__ node64, const uint32_t *status) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t eb = status[STATUS_VEXP];
    const int k = eb ? (int)eb - (int)VEXP_BIAS : 0;
    const double x = v[i];
    node[i].v = __double2float_rn(ldexp(x, -k));
    node64[i].v = x;
}

// t = 0: exp(0 A) v = v.
__global__ void k_copy_v(const int32_t *__restrict__ entries, int64_t n_entries, int64_t n,
                         const NodeRec64 *__restrict__ node64, double *mean, double *sem, uint32_t *status) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_entries) return;
    const int64_t i = entries ? entries[e] : e;
    if (i < 0 || i >= n) {
        atomicOr(status, ST_BAD_ENTRY);
        mean[e] = QNAN;
        if (sem) sem[e] = QNAN;
        return;
    }
    mean[e] = node64[i].v;
    if (sem) sem[e] = 0.0;
}

// ---------------------------------------------------------------------------
// Forward form (Lemma 2, Theorem 2, Algorithm 2) on the plan of B = A^T.
//
// Start draw j ~ v_j / V by a two-level alias: groups of START_GROUP indices
// (the last one ragged) with sums S_g summed in index order, V = sum of the
// S_g in group order; a canonical Vose table over the S_g picks the group and
// one over the group's v_j picks the member.  One Philox block per start,
// counter {0, 0xFFFFFFFF, path}: words 0/1 pick the group, words 2/3 the
// member.  Walk events use counter {k, 0xFFFFFFFE, path}.  Each path deposits
// V W at its end state: exact integer counts when every potential is zero
// (W = 1, e.g. a CTMC generator), FP64 atomic sums of V W and (V W)^2
// otherwise.
// ---------------------------------------------------------------------------
constexpr int64_t START_GROUP = 1024;
constexpr uint32_t FWD_START_STREAM = 0xFFFFFFFFu;
constexpr uint32_t FWD_WALK_STREAM = 0xFFFFFFFEu;

struct FwdTables {
    const AliasEnt *top;  // [G]
    const AliasEnt *in;   // [n]
    int64_t n;
    uint64_t G;
    const double *V;      // device scalar
    const uint32_t *bad;  // device flag: v invalid
};

// Group sums in index order; flags negative / non-finite entries.
__global__ void k_group_sums(int64_t n, const double *__restrict__ v, double *__restrict__ S, uint32_t *bad) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t G = (n + START_GROUP - 1) / START_GROUP;
    if (g >= G) return;
    const int64_t lo = g * START_GROUP, hi = min(n, lo + START_GROUP);
    double s = 0.0;
    bool b = false;
    for (int64_t i = lo; i < hi; ++i) {
        const double x = v[i];
        if (!(x >= 0.0) || !isfinite(x)) b = true;
        s = __dadd_rn(s, x);
    }
    S[g] = s;
    if (b) atomicOr(bad, 1u);
}

// V = sum of the group sums (group order) and the top-level table (one thread).
__global__ void k_top_table(int64_t G, const double *__restrict__ S, AliasEnt *top, double *q, int32_t *stack,
                            double *V, uint32_t *bad) {
    double s = 0.0;
    for (int64_t g = 0; g < G; ++g) s = __dadd_rn(s, S[g]);
    *V = s;
    if (!(s > 0.0) || !isfinite(s) || *bad) {
        atomicOr(bad, 1u);
        for (int64_t g = 0; g < G; ++g) top[g] = AliasEnt{(int32_t)g, 0xFFFFFFFFu};
        return;
    }
    vose_build((int32_t)G, S, s, [](int32_t k) { return k; }, top, q, stack);
}

// Member tables, one warp per group (all-zero groups are never drawn).
__global__ void k_inner_tables(int64_t n, const double *__restrict__ v, const double *__restrict__ S, AliasEnt *in,
                               double *q, int32_t *stack) {
    const int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int64_t G = (n + START_GROUP - 1) / START_GROUP;
    if (g >= G) return;  // uniform across the warp
    const int64_t lo = g * START_GROUP;
    const int32_t d = (int32_t)(min(n, lo + START_GROUP) - lo);
    if (S[g] > 0.0) {
        vose_build_warp(d, v + lo, S[g], [lo](int32_t k) { return (int32_t)(lo + k); }, in + lo, q + lo, stack + lo,
                        lane);
    } else {
        for (int32_t k = lane; k < d; k += 32) in[lo + k] = AliasEnt{(int32_t)(lo + k), 0xFFFFFFFFu};
    }
}

__device__ __forceinline__ int32_t forward_start(const FwdTables &f, const WalkParams &a, uint64_t path) {
    const uint4 w = philox_rk(make_uint4(0u, FWD_START_STREAM, (uint32_t)path, (uint32_t)(path >> 32)), a);
    int64_t g = (int64_t)(((unsigned long long)w.x * f.G) >> 32);
    const AliasEnt tg = f.top[g];
    if (!(w.y < tg.thresh)) g = tg.alias_col;
    const int64_t lo = g * START_GROUP;
    const uint32_t d = (uint32_t)(min(f.n, lo + START_GROUP) - lo);
    int64_t j = lo + __umulhi(w.z, d);
    const AliasEnt tj = f.in[j];
    if (!(w.w < tj.thresh)) j = tj.alias_col;
    return (int32_t)j;
}

struct FwdOut {
    unsigned long long *count;  // [n], zero-potential plans
    double *sum1;               // [n] sum of V W
    double *sum2;               // [n] sum of (V W)^2
};

template <int MODE, bool WEIGHTED, bool F64, bool COUNT>
__global__ void __launch_bounds__(WALK_THREADS, F64 ? WALK_MIN_BLOCKS_F64 : WALK_MIN_BLOCKS_F32)
    k_walk_forward(const __grid_constant__ WalkParams a, const __grid_constant__ FwdTables f, FwdOut o) {
    using Q = P<F64>;
    using T = typename Q::T;
    const int lane = threadIdx.x & 31;
    const uint64_t wid = ((uint64_t)blockIdx.x * WALK_THREADS + threadIdx.x) >> 5;
    const uint64_t p_begin = wid * a.chunk_len;
    if (p_begin >= a.paths || *f.bad) return;  // uniform across the warp
    const uint32_t len = (uint32_t)(min(a.paths, p_begin + a.chunk_len) - p_begin);
    const uint64_t base = a.path_offset + p_begin;
    const T t0 = F64 ? (T)a.t64 : (T)a.t32;
    const double V = *f.V;
    uint32_t next = 32;
    uint32_t p = (uint32_t)lane;
    bool active = p < len;
    int32_t i0 = 0;
    T delta_start = (T)0;
    Walker<F64> w;
    auto start_path = [&]() {
        i0 = forward_start(f, a, base + p);
        w.rec = load_node(a.node, i0);
        w.j = i0; w.r = t0; w.acc = (T)0; w.k = 0;
        delta_start = Q::pot(w.rec, a.node64, i0);
        w.delta = delta_start;
    };
    if (active) start_path();
    uint32_t jumps = 0;
    const unsigned lt_mask = (1u << lane) - 1u;
    while (__any_sync(0xffffffffu, active)) {
        bool fin = false;
        if (active && advance<MODE, WEIGHTED, F64>(w, a, FWD_WALK_STREAM, base + p, nullptr, -1)) {
            fin = true;
            jumps += w.k;
            if (COUNT) {
                atomicAdd(o.count + w.j, 1ull);
            } else {
                const T L = final_logw<MODE, F64>(w, delta_start, a);
                const double y = V * exp((double)L);  // FP64: finite for any FP32 log-weight below ~709
                atomicAdd(o.sum1 + w.j, y);
                atomicAdd(o.sum2 + w.j, y * y);
            }
        }
        const unsigned fm = __ballot_sync(0xffffffffu, fin);
        if (fm) {
            if (fin) {
                p = next + (uint32_t)__popc(fm & lt_mask);
                active = p < len;
                if (active) start_path();
            }
            next += (uint32_t)__popc(fm);
        }
    }
    unsigned long long jl = jumps;
#pragma unroll
    for (int sh = 16; sh > 0; sh >>= 1) jl += __shfl_xor_sync(0xffffffffu, jl, sh);
    if (lane == 0) {
        unsigned long long *ctr = reinterpret_cast<unsigned long long *>(a.status + 2);
        atomicAdd(ctr, (unsigned long long)len);
        atomicAdd(ctr + 1, jl);
    }
}

// Total communicability TC(t) = 1^T exp(tA) 1 (Sec. 6): the forward paths of
// v = 1 (Theorem 2; V = n, start uniform through the same two-level table) with
// no deposit: TC = V E[W].  Each warp leaves one partial (shifted sums of W)
// for the chunk reduction.
template <int MODE, bool WEIGHTED, bool F64>
__global__ void __launch_bounds__(WALK_THREADS, F64 ? WALK_MIN_BLOCKS_F64 : WALK_MIN_BLOCKS_F32)
    k_walk_tc(const __grid_constant__ WalkParams a, const __grid_constant__ FwdTables f) {
    using Q = P<F64>;
    using T = typename Q::T;
    using Acc = typename std::conditional<F64, Acc64, Acc32>::type;
    const int lane = threadIdx.x & 31;
    const uint64_t wid = ((uint64_t)blockIdx.x * WALK_THREADS + threadIdx.x) >> 5;
    const uint64_t p_begin = wid * a.chunk_len;
    if (p_begin >= a.paths) return;  // uniform across the warp
    const uint32_t len = (uint32_t)(min(a.paths, p_begin + a.chunk_len) - p_begin);
    const uint64_t base = a.path_offset + p_begin;
    const T t0 = F64 ? (T)a.t64 : (T)a.t32;
    uint32_t next = 32;
    uint32_t p = (uint32_t)lane;
    bool active = p < len;
    int32_t i0 = 0;
    T delta_start = (T)0;
    Walker<F64> w;
    auto start_path = [&]() {
        i0 = forward_start(f, a, base + p);
        w.rec = load_node(a.node, i0);
        w.j = i0; w.r = t0; w.acc = (T)0; w.k = 0;
        delta_start = Q::pot(w.rec, a.node64, i0);
        w.delta = delta_start;
    };
    if (active) start_path();
    Acc acc;
    uint32_t jumps = 0;
    const unsigned lt_mask = (1u << lane) - 1u;
    while (__any_sync(0xffffffffu, active)) {
        bool fin = false;
        if (active && advance<MODE, WEIGHTED, F64>(w, a, FWD_WALK_STREAM, base + p, nullptr, -1)) {
            fin = true;
            jumps += w.k;
            acc.add(final_logw<MODE, F64>(w, delta_start, a), (T)1);
        }
        const unsigned fm = __ballot_sync(0xffffffffu, fin);
        if (fm) {
            if (fin) {
                p = next + (uint32_t)__popc(fm & lt_mask);
                active = p < len;
                if (active) start_path();
            }
            next += (uint32_t)__popc(fm);
        }
    }
    unsigned long long jl = jumps;
#pragma unroll
    for (int sh = 16; sh > 0; sh >>= 1) jl += __shfl_xor_sync(0xffffffffu, jl, sh);
    double S1, S2, Mw;
    acc.warp_merge(S1, S2, Mw);
    if (lane == 0) {
        unsigned long long *ctr = reinterpret_cast<unsigned long long *>(a.status + 2);
        atomicAdd(ctr, (unsigned long long)len);
        atomicAdd(ctr + 1, jl);
        a.partials[wid] = Partial{S1, S2, Mw};
    }
}

__global__ void k_fill(int64_t n, double *x, double value) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] = value;
}

// All warp partials of a TC call merged by one block: the common shift (max),
// then the rescaled sums in a fixed thread-strided order and tree; the result
// (V mean, V SE) with V = *Vp.
__global__ void __launch_bounds__(WALK_THREADS) k_reduce_tc(const Partial *__restrict__ part, uint32_t np, double M,
                                                            const double *Vp, double *tc, double *sem,
                                                            uint32_t *status) {
    __shared__ double sh[WARPS_PER_BLOCK][2];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double m = -INFINITY;
    for (uint32_t c = threadIdx.x; c < np; c += WALK_THREADS) m = fmax(m, part[c].m);
    m = warp_max(m);
    if (lane == 0) sh[warp][0] = m;
    __syncthreads();
    m = -INFINITY;
    for (int w = 0; w < WARPS_PER_BLOCK; ++w) m = fmax(m, sh[w][0]);
    __syncthreads();
    double s1 = 0.0, s2 = 0.0;
    for (uint32_t c = threadIdx.x; c < np; c += WALK_THREADS) {
        const Partial q = part[c];
        const double sc = q.m == -INFINITY ? 0.0 : exp(q.m - m);
        s1 += sc * q.s1;
        s2 += sc * sc * q.s2;
    }
    s1 = warp_sum(s1);
    s2 = warp_sum(s2);
    if (lane == 0) {
        sh[warp][0] = s1;
        sh[warp][1] = s2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < WARPS_PER_BLOCK; ++w) {
            a += sh[w][0];
            b += sh[w][1];
        }
        double mean, se;
        finish_entry(a, b, m, M, 1.0, &mean, &se, status);
        const double V = *Vp;
        *tc = V * mean;
        if (sem) *sem = V * se;
    }
}

// x_i = (sum of V W 1{end = i}) / M and its standard error.
__global__ void k_forward_finish(int64_t n, FwdOut o, const double *Vp, const uint32_t *bad, double M, double *x,
                                 double *sem, uint32_t *status) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (*bad) {
        x[i] = QNAN;
        if (sem) sem[i] = QNAN;
        if (i == 0) atomicOr(status, ST_BAD_V);
        return;
    }
    double s1, s2;
    if (o.count) {
        const double c = (double)o.count[i];
        const double V = *Vp;
        s1 = V * c;
        s2 = V * V * c;
    } else {
        s1 = o.sum1[i];
        s2 = o.sum2[i];
    }
    const double mu = s1 / M;
    double var = M > 1.0 ? (s2 - s1 * mu) / (M - 1.0) : 0.0;
    if (var < 0.0) var = 0.0;
    x[i] = mu;
    if (sem) sem[i] = sqrt(var / M);
    if (!isfinite(mu) || !isfinite(var)) atomicOr(status, ST_OVERFLOW);
}

template <int MODE, bool WEIGHTED, bool F64>
__global__ void __launch_bounds__(WALK_THREADS) k_trace_forward(const __grid_constant__ WalkParams a,
                                                               const __grid_constant__ FwdTables f,
                                                               uint64_t first_path, uint32_t count, int32_t *start,
                                                               int32_t *end, uint32_t *njumps, uint64_t *hash,
                                                               double *logw) {
    using Q = P<F64>;
    using T = typename Q::T;
    const uint32_t q = blockIdx.x * WALK_THREADS + threadIdx.x;
    if (q >= count) return;
    if (*f.bad) {
        if (q == 0) atomicOr(a.status, ST_BAD_V);
        return;
    }
    const uint64_t path = first_path + q;
    const int32_t i = forward_start(f, a, path);
    Walker<F64> w;
    w.rec = load_node(a.node, i);
    const T delta_start = Q::pot(w.rec, a.node64, i);
    w.j = i; w.r = F64 ? (T)a.t64 : (T)a.t32; w.acc = (T)0; w.delta = delta_start; w.k = 0;
    uint64_t h = (FNV_OFFSET ^ (uint64_t)(uint32_t)i) * FNV_PRIME;
    if (a.t64 != 0.0) {
        while (!advance<MODE, WEIGHTED, F64>(w, a, FWD_WALK_STREAM, path, nullptr, -1))
            h = (h ^ (uint64_t)(uint32_t)w.j) * FNV_PRIME;
    }
    start[q] = i;
    end[q] = w.j;
    njumps[q] = w.k;
    hash[q] = h;
    logw[q] = a.t64 != 0.0 ? (double)final_logw<MODE, F64>(w, delta_start, a) : 0.0;
}

template <bool F64, bool WEIGHTED>
cudaError_t launch_lanes_mode(int mode, unsigned grid, const WalkParams &p, cudaStream_t st) {
    switch (mode) {
        case MCX_EXACT: k_walk_lanes<MCX_EXACT, WEIGHTED, F64><<<grid, WALK_THREADS, 0, st>>>(p); break;
        case MCX_STRANG: k_walk_lanes<MCX_STRANG, WEIGHTED, F64><<<grid, WALK_THREADS, 0, st>>>(p); break;
        default: k_walk_lanes<MCX_LIE, WEIGHTED, F64><<<grid, WALK_THREADS, 0, st>>>(p); break;
    }
    return cudaGetLastError();
}

template <bool F64, bool WEIGHTED>
cudaError_t launch_walk_mode(int mode, unsigned grid, const WalkParams &p, cudaStream_t st) {
    switch (mode) {
        case MCX_EXACT: k_walk<MCX_EXACT, WEIGHTED, F64><<<grid, WALK_THREADS, 0, st>>>(p); break;
        case MCX_STRANG: k_walk<MCX_STRANG, WEIGHTED, F64><<<grid, WALK_THREADS, 0, st>>>(p); break;
        default: k_walk<MCX_LIE, WEIGHTED, F64><<<grid, WALK_THREADS, 0, st>>>(p); break;
    }
    return cudaGetLastError();
}

template <bool F64, bool WEIGHTED>
cudaError_t launch_trace_mode(int mode, unsigned grid, const WalkParams &p, int32_t i, uint64_t first,
                              uint32_t count, int32_t *end, uint32_t *nj, uint64_t *h, double *lw, cudaStream_t st) {
    switch (mode) {
        case MCX_EXACT: k_trace<MCX_EXACT, WEIGHTED, F64><<<grid, WALK_THREADS, 0, st>>>(p, i, first, count, end, nj, h, lw); break;
        case MCX_STRANG: k_trace<MCX_STRANG, WEIGHTED, F64><<<grid, WALK_THREADS, 0, st>>>(p, i, first, count, end, nj, h, lw); break;
        default: k_trace<MCX_LIE, WEIGHTED, F64><<<grid, WALK_THREADS, 0, st>>>(p, i, first, count, end, nj, h, lw); break;
    }
    return cudaGetLastError();
}


}  // namespace

cudaError_t launch_pack_v(mcx_plan *plan, const double *v, cudaStream_t st) {
    if (plan->n == 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(plan->status + STATUS_VEXP, 0, 4, st);
    if (e != cudaSuccess) return e;
    const unsigned blocks = (unsigned)std::min<int64_t>((plan->n + 255) / 256, 152 * 8);
    k_v_exponent<<<blocks, 256, 0, st>>>(plan->n, v, plan->status);
    k_pack_v<<<(unsigned)((plan->n + 255) / 256), 256, 0, st>>>(plan->n, v, plan->node, plan->node64, plan->status);
    return cudaGetLastError();
}

namespace {

// Chunking of an estimate over warps: at least 1024 paths per warp, and enough
// warps to fill the GPU several times over (152 SMs x 64 resident warps x 8
// waves); chunk lengths are multiples of 32 and below 2^30 paths (32-bit chunk
// offsets).  Shared by mcx_estimate and mcx_estimate_noalloc, whose results
// are therefore identical.
struct Chunking {
    uint64_t chunk;     // paths per warp
    uint64_t cpe;       // chunks per entry
    uint64_t n_chunks;  // n_entries * cpe
};

Chunking estimate_chunking(const EstimateArgs &a) {
    const uint64_t target_warps = 152ull * 64ull * 8ull;
    uint64_t cpe = (target_warps + (uint64_t)a.n_entries - 1) / (uint64_t)a.n_entries;
    const uint64_t max_cpe = (a.paths + 1023) / 1024;
    if (cpe > max_cpe) cpe = max_cpe;
    if (cpe < 1) cpe = 1;
    if ((a.paths + cpe - 1) / cpe > (1ull << 30)) cpe = (a.paths + (1ull << 30) - 1) >> 30;
    uint64_t chunk = (a.paths + cpe - 1) / cpe;
    chunk = (chunk + 31) / 32 * 32;
    cpe = (a.paths + chunk - 1) / chunk;
    return Chunking{chunk, cpe, (uint64_t)a.n_entries * cpe};
}

// Walk parameters of an estimate (t > 0).
WalkParams estimate_params(mcx_plan *plan, const EstimateArgs &a) {
    WalkParams p = make_params(plan, a.t, a.mode == MCX_EXACT ? 1 : a.nsteps, a.seed);
    p.entries = a.entries;
    p.n_entries = a.n_entries;
    p.paths = a.paths;
    p.path_offset = a.path_offset;
    p.mean = a.mean;
    p.sem = a.sem;
    return p;
}

// t = 0: the entries of v.
cudaError_t launch_copy_v(mcx_plan *plan, const EstimateArgs &a, cudaStream_t st) {
    k_copy_v<<<(unsigned)((a.n_entries + 255) / 256), 256, 0, st>>>(a.entries, a.n_entries, plan->n, plan->node64,
                                                                      a.mean, a.sem, plan->status);
    return cudaGetLastError();
}

// One lane per entry (at most LANE_MODE_MAX_PATHS paths): no partials.
cudaError_t launch_lanes(mcx_plan *plan, const EstimateArgs &a, cudaStream_t st) {
    const WalkParams p = estimate_params(plan, a);
    const unsigned grid = (unsigned)((a.n_entries + WALK_THREADS - 1) / WALK_THREADS);
    const bool weighted = plan->weighted_rows > 0;
    if (a.precision == MCX_FP64)
        return weighted ? launch_lanes_mode<true, true>(a.mode, grid, p, st)
                        : launch_lanes_mode<true, false>(a.mode, grid, p, st);
    return weighted ? launch_lanes_mode<false, true>(a.mode, grid, p, st)
                    : launch_lanes_mode<false, false>(a.mode, grid, p, st);
}

// Warp per (entry, chunk) and, when entries span several chunks, the chunk
// merge over `partials` (c.n_chunks of them).
cudaError_t launch_chunks(mcx_plan *plan, const EstimateArgs &a, const Chunking &c, Partial *partials,
                          cudaStream_t st) {
    WalkParams p = estimate_params(plan, a);
    p.chunk_len = c.chunk;
    p.chunks_per_entry = (uint32_t)c.cpe;
    p.partials = partials;
    const unsigned grid = (unsigned)((c.n_chunks + WARPS_PER_BLOCK - 1) / WARPS_PER_BLOCK);
    const bool weighted = plan->weighted_rows > 0;
    cudaError_t e;
    if (a.precision == MCX_FP64) {
        e = weighted ? launch_walk_mode<true, true>(a.mode, grid, p, st) : launch_walk_mode<true, false>(a.mode, grid, p, st);
    } else {
        e = weighted ? launch_walk_mode<false, true>(a.mode, grid, p, st) : launch_walk_mode<false, false>(a.mode, grid, p, st);
    }
    if (e != cudaSuccess) return e;
    if (c.cpe > 1) {
        const unsigned g2 = (unsigned)((a.n_entries + WARPS_PER_BLOCK - 1) / WARPS_PER_BLOCK);
        k_reduce_chunks<<<g2, WALK_THREADS, 0, st>>>(partials, a.n_entries, (uint32_t)c.cpe, (double)a.paths,
                                                    a.precision != MCX_FP64, a.mean, a.sem, plan->status);
        e = cudaGetLastError();
    }
    return e;
}

}  // namespace

cudaError_t launch_estimate(mcx_plan *plan, const EstimateArgs &a, cudaStream_t st) {
    if (a.n_entries == 0) return cudaSuccess;
    if (a.t == 0.0) return launch_copy_v(plan, a, st);
    if (a.paths <= LANE_MODE_MAX_PATHS) return launch_lanes(plan, a, st);
    const Chunking c = estimate_chunking(a);
    if (c.cpe > 1) {
        const size_t need = sizeof(Partial) * (size_t)c.n_chunks;
        if (plan->scratch_bytes < need) {
            dev_free(plan->scratch);
            plan->scratch = nullptr;
            plan->scratch_bytes = 0;
            cudaError_t e = dev_malloc(&plan->scratch, need);
            if (e != cudaSuccess) return e;
            plan->scratch_bytes = need;
        }
    }
    return launch_chunks(plan, a, c, static_cast<Partial *>(plan->scratch), st);
}

namespace {

// Forward scratch: S[G], top[G], in[n], q[max(n,G)], stack[max(n,G)], V, bad, deposits[2n].
struct FwdScratch {
    double *S;
    AliasEnt *top;
    AliasEnt *in;
    double *q;
    int32_t *stack;
    double *V;
    uint32_t *bad;
    double *dep;  // 2n doubles (sum1, sum2) or n u64 counts
};

cudaError_t fwd_scratch(mcx_plan *plan, FwdScratch *fs) {
    const int64_t n = plan->n;
    const int64_t G = (n + START_GROUP - 1) / START_GROUP;
    const int64_t m = n > G ? n : G;
    auto seg = [](size_t bytes) { return (bytes + 255) / 256 * 256; };
    const size_t need = seg(16 * (size_t)n) + seg(8 * (size_t)G) + seg(8 * (size_t)G) + seg(8 * (size_t)n) +
                        seg(8 * (size_t)m) + seg(4 * (size_t)m) + seg(8) + seg(8);
    if (plan->fwd_bytes < need) {
        dev_free(plan->fwd);
        plan->fwd = nullptr;
        plan->fwd_bytes = 0;
        plan->fwd_ones = false;
        cudaError_t e = dev_malloc(&plan->fwd, need);
        if (e != cudaSuccess) return e;
        plan->fwd_bytes = need;
    }
    char *b = static_cast<char *>(plan->fwd);
    auto take = [&b](size_t bytes) {
        char *r = b;
        b += (bytes + 255) / 256 * 256;
        return r;
    };
    fs->dep = reinterpret_cast<double *>(take(16 * (size_t)n));
    fs->S = reinterpret_cast<double *>(take(8 * (size_t)G));
    fs->top = reinterpret_cast<AliasEnt *>(take(8 * (size_t)G));
    fs->in = reinterpret_cast<AliasEnt *>(take(8 * (size_t)n));
    fs->q = reinterpret_cast<double *>(take(8 * (size_t)m));
    fs->stack = reinterpret_cast<int32_t *>(take(4 * (size_t)m));
    fs->V = reinterpret_cast<double *>(take(8));
    fs->bad = reinterpret_cast<uint32_t *>(take(8));
    return cudaSuccess;
}

// Build the two-level start tables on `st`; fills the FwdTables view.
// the tables in the forward scratch as the walkers see them
FwdTables start_view(const mcx_plan *plan, const FwdScratch &fs) {
    FwdTables f;
    f.top = fs.top;
    f.in = fs.in;
    f.n = plan->n;
    f.G = (uint64_t)((plan->n + START_GROUP - 1) / START_GROUP);
    f.V = fs.V;
    f.bad = fs.bad;
    return f;
}

cudaError_t build_start_tables(mcx_plan *plan, const double *v, const FwdScratch &fs, FwdTables *f, cudaStream_t st) {
    const int64_t n = plan->n;
    const int64_t G = (n + START_GROUP - 1) / START_GROUP;
    plan->fwd_ones = false;
    cudaError_t e = cudaMemsetAsync(fs.bad, 0, 4, st);
    if (e != cudaSuccess) return e;
    const unsigned gb = (unsigned)((G + 127) / 128);
    k_group_sums<<<gb, 128, 0, st>>>(n, v, fs.S, fs.bad);
    k_top_table<<<1, 1, 0, st>>>(G, fs.S, fs.top, fs.q, fs.stack, fs.V, fs.bad);
    k_inner_tables<<<(unsigned)((G + 3) / 4), 128, 0, st>>>(n, v, fs.S, fs.in, fs.q, fs.stack);  // warp per group
    *f = start_view(plan, fs);
    return cudaGetLastError();
}

template <bool F64, bool WEIGHTED, bool COUNT>
void launch_fwd(int mode, unsigned grid, const WalkParams &p, const FwdTables &f, const FwdOut &o, cudaStream_t st) {
    switch (mode) {
        case MCX_EXACT: k_walk_forward<MCX_EXACT, WEIGHTED, F64, COUNT><<<grid, WALK_THREADS, 0, st>>>(p, f, o); break;
        case MCX_STRANG: k_walk_forward<MCX_STRANG, WEIGHTED, F64, COUNT><<<grid, WALK_THREADS, 0, st>>>(p, f, o); break;
        default: k_walk_forward<MCX_LIE, WEIGHTED, F64, COUNT><<<grid, WALK_THREADS, 0, st>>>(p, f, o); break;
    }
}

template <bool F64, bool WEIGHTED>
void launch_fwd_trace(int mode, unsigned grid, const WalkParams &p, const FwdTables &f, uint64_t first, uint32_t count,
                      int32_t *start, int32_t *end, uint32_t *nj, uint64_t *h, double *lw, cudaStream_t st) {
    switch (mode) {
        case MCX_EXACT: k_trace_forward<MCX_EXACT, WEIGHTED, F64><<<grid, WALK_THREADS, 0, st>>>(p, f, first, count, start, end, nj, h, lw); break;
        case MCX_STRANG: k_trace_forward<MCX_STRANG, WEIGHTED, F64><<<grid, WALK_THREADS, 0, st>>>(p, f, first, count, start, end, nj, h, lw); break;
        default: k_trace_forward<MCX_LIE, WEIGHTED, F64><<<grid, WALK_THREADS, 0, st>>>(p, f, first, count, start, end, nj, h, lw); break;
    }
}

}  // namespace

cudaError_t launch_estimate_forward(mcx_plan *plan, const double *v, double t, int mode, int nsteps, uint64_t paths,
                                    uint64_t seed, uint64_t path_offset, int precision, double *x, double *sem,
                                    cudaStream_t st) {
    const int64_t n = plan->n;
    if (n == 0) return cudaSuccess;
    FwdScratch fs;
    cudaError_t e = fwd_scratch(plan, &fs);
    if (e != cudaSuccess) return e;
    FwdTables f;
    if ((e = build_start_tables(plan, v, fs, &f, st)) != cudaSuccess) return e;
    WalkParams p = make_params(plan, t, mode == MCX_EXACT ? 1 : nsteps, seed);
    p.paths = paths;
    p.path_offset = path_offset;
    const uint64_t target_warps = 152ull * 64ull * 8ull;
    uint64_t chunk = (paths + target_warps - 1) / target_warps;
    if (chunk < 256) chunk = 256;
    if (chunk > (1ull << 30)) chunk = 1ull << 30;
    chunk = (chunk + 31) / 32 * 32;
    p.chunk_len = chunk;
    const uint64_t n_warps = (paths + chunk - 1) / chunk;
    const unsigned grid = (unsigned)((n_warps + WARPS_PER_BLOCK - 1) / WARPS_PER_BLOCK);
    const bool count = plan->zero_potential;
    FwdOut o{};
    if (count) {
        o.count = reinterpret_cast<unsigned long long *>(fs.dep);
        e = cudaMemsetAsync(fs.dep, 0, 8 * (size_t)n, st);
    } else {
        o.sum1 = fs.dep;
        o.sum2 = fs.dep + n;
        e = cudaMemsetAsync(fs.dep, 0, 16 * (size_t)n, st);
    }
    if (e != cudaSuccess) return e;
    const bool wgt = plan->weighted_rows > 0;
    if (paths > 0) {
        if (precision == MCX_FP64) {
            if (count) { if (wgt) launch_fwd<true, true, true>(mode, grid, p, f, o, st); else launch_fwd<true, false, true>(mode, grid, p, f, o, st); }
            else { if (wgt) launch_fwd<true, true, false>(mode, grid, p, f, o, st); else launch_fwd<true, false, false>(mode, grid, p, f, o, st); }
        } else {
            if (count) { if (wgt) launch_fwd<false, true, true>(mode, grid, p, f, o, st); else launch_fwd<false, false, true>(mode, grid, p, f, o, st); }
            else { if (wgt) launch_fwd<false, true, false>(mode, grid, p, f, o, st); else launch_fwd<false, false, false>(mode, grid, p, f, o, st); }
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    k_forward_finish<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, o, fs.V, fs.bad, (double)paths, x, sem,
                                                                   plan->status);
    return cudaGetLastError();
}

template <bool F64, bool WEIGHTED>
void launch_tc_kernel(int mode, unsigned grid, const WalkParams &p, const FwdTables &f, cudaStream_t st) {
    switch (mode) {
        case MCX_EXACT: k_walk_tc<MCX_EXACT, WEIGHTED, F64><<<grid, WALK_THREADS, 0, st>>>(p, f); break;
        case MCX_STRANG: k_walk_tc<MCX_STRANG, WEIGHTED, F64><<<grid, WALK_THREADS, 0, st>>>(p, f); break;
        default: k_walk_tc<MCX_LIE, WEIGHTED, F64><<<grid, WALK_THREADS, 0, st>>>(p, f); break;
    }
}

cudaError_t launch_total_communicability(mcx_plan *plan, double t, int mode, int nsteps, uint64_t paths,
                                         uint64_t seed, uint64_t path_offset, int precision, double *tc, double *sem,
                                         cudaStream_t st) {
    const int64_t n = plan->n;
    FwdScratch fs;
    cudaError_t e = fwd_scratch(plan, &fs);
    if (e != cudaSuccess) return e;
    // the start tables of v = 1 are built once and kept until another forward call replaces them
    FwdTables f = start_view(plan, fs);
    if (!plan->fwd_ones) {
        double *ones = fs.dep;  // the deposit area is free in this mode
        k_fill<<<(unsigned)std::min<int64_t>((n + 255) / 256, 152 * 32), 256, 0, st>>>(n, ones, 1.0);
        if ((e = build_start_tables(plan, ones, fs, &f, st)) != cudaSuccess) return e;
        plan->fwd_ones = true;
    }
    WalkParams p = make_params(plan, t, mode == MCX_EXACT ? 1 : nsteps, seed);
    p.paths = paths;
    p.path_offset = path_offset;
    const uint64_t target_warps = 152ull * 64ull * 8ull;
    uint64_t chunk = (paths + target_warps - 1) / target_warps;
    if (chunk < 256) chunk = 256;
    if (chunk > (1ull << 30)) chunk = 1ull << 30;
    chunk = (chunk + 31) / 32 * 32;
    p.chunk_len = chunk;
    const uint64_t n_warps = (paths + chunk - 1) / chunk;
    const size_t need = sizeof(Partial) * (size_t)n_warps;
    if (plan->scratch_bytes < need) {
        dev_free(plan->scratch);
        plan->scratch = nullptr;
        plan->scratch_bytes = 0;
        if ((e = dev_malloc(&plan->scratch, need)) != cudaSuccess) return e;
        plan->scratch_bytes = need;
    }
    p.partials = static_cast<Partial *>(plan->scratch);
    const unsigned grid = (unsigned)((n_warps + WARPS_PER_BLOCK - 1) / WARPS_PER_BLOCK);
    const bool wgt = plan->weighted_rows > 0;
    if (precision == MCX_FP64) {
        if (wgt) launch_tc_kernel<true, true>(mode, grid, p, f, st); else launch_tc_kernel<true, false>(mode, grid, p, f, st);
    } else {
        if (wgt) launch_tc_kernel<false, true>(mode, grid, p, f, st); else launch_tc_kernel<false, false>(mode, grid, p, f, st);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_reduce_tc<<<1, WALK_THREADS, 0, st>>>(p.partials, (uint32_t)n_warps, (double)paths, fs.V, tc, sem,
                                             plan->status);
    return cudaGetLastError();
}

cudaError_t launch_trace_forward(mcx_plan *plan, const double *v, double t, int mode, int nsteps, uint64_t seed,
                                 uint64_t first_path, uint32_t count, int precision, int32_t *start, int32_t *end,
                                 uint32_t *njumps, uint64_t *hash, double *logw, cudaStream_t st) {
    if (count == 0 || plan->n == 0) return cudaSuccess;
    FwdScratch fs;
    cudaError_t e = fwd_scratch(plan, &fs);
    if (e != cudaSuccess) return e;
    FwdTables f;
    if ((e = build_start_tables(plan, v, fs, &f, st)) != cudaSuccess) return e;
    WalkParams p = make_params(plan, t, mode == MCX_EXACT ? 1 : nsteps, seed);
    const unsigned grid = (count + WALK_THREADS - 1) / WALK_THREADS;
    const bool wgt = plan->weighted_rows > 0;
    if (precision == MCX_FP64) {
        if (wgt) launch_fwd_trace<true, true>(mode, grid, p, f, first_path, count, start, end, njumps, hash, logw, st);
        else launch_fwd_trace<true, false>(mode, grid, p, f, first_path, count, start, end, njumps, hash, logw, st);
    } else {
        if (wgt) launch_fwd_trace<false, true>(mode, grid, p, f, first_path, count, start, end, njumps, hash, logw, st);
        else launch_fwd_trace<false, false>(mode, grid, p, f, first_path, count, start, end, njumps, hash, logw, st);
    }
    return cudaGetLastError();
}

cudaError_t launch_trace(mcx_plan *plan, double t, int mode, int nsteps, int32_t entry, uint64_t seed,
                         uint64_t first_path, uint32_t count, int precision, int32_t *end, uint32_t *njumps,
                         uint64_t *hash, double *logw, cudaStream_t st) {
    if (count == 0) return cudaSuccess;
    const unsigned grid = (count + WALK_THREADS - 1) / WALK_THREADS;
    if (t == 0.0) {
        k_trace_t0<<<grid, WALK_THREADS, 0, st>>>(entry, count, end, njumps, hash, logw);
        return cudaGetLastError();
    }
    WalkParams p = make_params(plan, t, mode == MCX_EXACT ? 1 : nsteps, seed);
    const bool weighted = plan->weighted_rows > 0;
    if (precision == MCX_FP64) {
        return weighted ? launch_trace_mode<true, true>(mode, grid, p, entry, first_path, count, end, njumps, hash, logw, st)
                        : launch_trace_mode<true, false>(mode, grid, p, entry, first_path, count, end, njumps, hash, logw, st);
    }
    return weighted ? launch_trace_mode<false, true>(mode, grid, p, entry, first_path, count, end, njumps, hash, logw, st)
                    : launch_trace_mode<false, false>(mode, grid, p, entry, first_path, count, end, njumps, hash, logw, st);
}

// ---------------------------------------------------------------------------
// Estimate that allocates nothing (mcx_estimate_noalloc).
//
// mcx_estimate keeps its per-chunk partial sums in plan scratch that it grows
// with cudaMalloc on demand.  This variant runs the same kernels but keeps the
// partials in the fixed array below, compiled into the library: every GPU that
// loads the library holds NOALLOC_MAX_PARTIALS * 24 bytes (3 MiB) of it until
// the process exits.  All calls share the array and it keeps the last call's
// contents; nothing in it needs to start at zero, because each call writes
// every slot it reads (k_walk writes one partial per chunk before
// k_reduce_chunks reads it).  Two calls that overlap on the GPU (different
// streams, or different threads without ordering) race on the array.
// ---------------------------------------------------------------------------
constexpr uint64_t NOALLOC_MAX_PARTIALS = 1ull << 17;
static __device__ __align__(256) Partial g_noalloc_partials[NOALLOC_MAX_PARTIALS];

namespace {

constexpr int NOALLOC_MAX_DEVICES = 64;
std::mutex g_noalloc_mutex;
Partial *g_noalloc_ptr[NOALLOC_MAX_DEVICES];

// Device address of g_noalloc_partials on the current device.  In host code the
// array's name only stands for it, so the address is looked up per device (with
// that device current) and cached once the lookup has succeeded; a failed
// lookup is returned and tried again on the next call.
cudaError_t noalloc_partials(Partial **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (g_noalloc_ptr[dev] == nullptr) {
        void *ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_noalloc_partials);
        if (e != cudaSuccess) return e;
        g_noalloc_ptr[dev] = static_cast<Partial *>(ptr);
    }
    *out = g_noalloc_ptr[dev];
    return cudaSuccess;
}

}  // namespace

uint64_t noalloc_max_partials() { return NOALLOC_MAX_PARTIALS; }

cudaError_t launch_estimate_noalloc(mcx_plan *plan, const double *v, const EstimateArgs &a, cudaStream_t st,
                                    bool *too_large) {
    *too_large = false;
    if (a.n_entries == 0) return cudaSuccess;
    const bool walk = a.t != 0.0 && a.paths > LANE_MODE_MAX_PATHS;
    const Chunking c = estimate_chunking(a);
    if (walk && c.cpe > 1 && c.n_chunks > NOALLOC_MAX_PARTIALS) {
        *too_large = true;  // rejected before anything is enqueued
        return cudaSuccess;
    }
    Partial *partials = nullptr;
    cudaError_t e = noalloc_partials(&partials);
    if (e != cudaSuccess) return e;
    if ((e = launch_pack_v(plan, v, st)) != cudaSuccess) return e;
    if (a.t == 0.0) return launch_copy_v(plan, a, st);
    if (!walk) return launch_lanes(plan, a, st);
    return launch_chunks(plan, a, c, partials, st);
}

}  // namespace mcx
