// Batching: many forward problems (Lemma 2, Theorem 2, Algorithm 2) in one
// persistent launch replayed from a CUDA graph, with an autotuned schedule.
//
// Layout.  The problems' plan matrices B_b (= A_b^T) are placed on the
// diagonal of one block-diagonal plan; block b starts at state off_b, a
// multiple of 1024, and the states between blocks are isolated padding (never
// drawn, never reached).  Start draws j ~ v_b / V_b use the two-level alias of
// the single-problem forward form per problem: groups of 1024 states inside
// the block (the last one ragged at the block's true end), a Vose table over
// the problem's group sums and one inside each group; so a batched
// (problem, time) pair with path indices pt * 2^40 + p draws exactly the
// paths of a single-problem forward run of that problem with path_offset
// pt * 2^40.
//
// Schedule.  The (problem, time) pairs are cut into work items of `chunk`
// paths; items are ordered by estimated cost per item, largest first
// (longest-processing-time order; cost ~ paths x (1 + t x mean jump rate));
// a persistent grid of warps takes items from an atomic counter.  Each warp
// runs its item's paths (with lane refill, or a fixed share per lane) and
// deposits at the end states: exact counts when every potential is zero
// (W = 1), FP64 sums otherwise.  The counter reset, deposit reset, walk and
// finish are captured once into a CUDA graph; each run only updates the walk
// node's seed.  The autotuner times the (lane refill, chunk, blocks per SM)
// settings on a sample of the items and keeps the fastest, cached by
// problem-set signature in a small JSON file.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <new>
#include <string>
#include <vector>

#include "launch.h"
#include "tune_cache.h"
#include "walker.cuh"

namespace mcx {
namespace {

constexpr int64_t BGROUP = 1024;

struct BatchPT {
    int64_t off;        // first global state of the problem
    int64_t n;          // states of the problem
    int64_t g0;         // first global start group
    int64_t G;          // groups of the problem
    uint64_t paths;     // forward paths for this time
    uint64_t path_base; // pt << 40
    int64_t dep;        // first deposit / output slot
    int32_t problem;
    int32_t tidx;
    double t;
};

struct BatchItem {
    uint32_t pt;
    uint32_t chunk;
};

struct BatchArgs {
    const BatchPT *pts;
    const BatchItem *items;
    uint32_t n_items;
    uint32_t chunk_len;
    unsigned int *next_item;
    const AliasEnt *top;        // per-problem top tables at [g0, g0 + G), local group ids
    const AliasEnt *in;         // member tables, global state ids
    const double *V;            // [problems]
    const uint32_t *bad;        // v invalid somewhere
    unsigned long long *count;  // [slots] (zero potential)
    double *sum1, *sum2;        // [slots] (otherwise)
};

__global__ void k_bgroup_sums(int64_t ngroups, const int32_t *__restrict__ gprob, const BatchPT *__restrict__ pbase,
                              const double *__restrict__ v, double *__restrict__ S, uint32_t *bad) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= ngroups) return;
    const int32_t b = gprob[g];
    if (b < 0) {
        S[g] = 0.0;
        return;
    }
    const BatchPT p = pbase[b];
    const int64_t lo = g * BGROUP, hi = min(p.off + p.n, lo + BGROUP);
    double s = 0.0;
    bool bd = false;
    for (int64_t i = lo; i < hi; ++i) {
        const double x = v[i];
        if (!(x >= 0.0) || !isfinite(x)) bd = true;
        s = __dadd_rn(s, x);
    }
    S[g] = s;
    if (bd) atomicOr(bad, 1u);
}

// One thread per problem: V_b = sum of its group sums (group order), top-level Vose.
__global__ void k_btop(int32_t problems, const BatchPT *__restrict__ pbase, const double *__restrict__ S,
                       AliasEnt *top, double *q, int32_t *stack, double *V, uint32_t *bad) {
    const int32_t b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= problems) return;
    const BatchPT p = pbase[b];
    double s = 0.0;
    for (int64_t g = 0; g < p.G; ++g) s = __dadd_rn(s, S[p.g0 + g]);
    V[b] = s;
    if (!(s > 0.0) || !isfinite(s)) {
        atomicOr(bad, 1u);
        for (int64_t g = 0; g < p.G; ++g) top[p.g0 + g] = AliasEnt{(int32_t)g, 0xFFFFFFFFu};
        return;
    }
    vose_build((int32_t)p.G, S + p.g0, s, [](int32_t k) { return k; }, top + p.g0, q + p.g0, stack + p.g0);
}

// One warp per group: member table over the group's states (true end of the block).
__global__ void k_binner(int64_t ngroups, const int32_t *__restrict__ gprob, const BatchPT *__restrict__ pbase,
                         const double *__restrict__ v, const double *__restrict__ S, AliasEnt *in, double *q,
                         int32_t *stack) {
    const int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (g >= ngroups) return;  // uniform across the warp
    const int32_t b = gprob[g];
    if (b < 0) return;
    const BatchPT p = pbase[b];
    const int64_t lo = g * BGROUP;
    const int32_t d = (int32_t)(min(p.off + p.n, lo + BGROUP) - lo);
    if (S[g] > 0.0) {
        vose_build_warp(d, v + lo, S[g], [lo](int32_t k) { return (int32_t)(lo + k); }, in + lo, q + lo, stack + lo,
                        lane);
    } else {
        for (int32_t k = lane; k < d; k += 32) in[lo + k] = AliasEnt{(int32_t)(lo + k), 0xFFFFFFFFu};
    }
}

__device__ __forceinline__ int32_t batch_start(const BatchArgs &b, const BatchPT &p, const WalkParams &a,
                                               uint64_t path) {
    const uint4 w = philox_rk(make_uint4(0u, 0xFFFFFFFFu, (uint32_t)path, (uint32_t)(path >> 32)), a);
    int64_t g = (int64_t)(((unsigned long long)w.x * (unsigned long long)p.G) >> 32);
    const AliasEnt tg = b.top[p.g0 + g];
    if (!(w.y < tg.thresh)) g = tg.alias_col;
    const int64_t lo = (p.g0 + g) * BGROUP;
    const uint32_t d = (uint32_t)(min(p.off + p.n, lo + BGROUP) - lo);
    int64_t j = lo + __umulhi(w.z, d);
    const AliasEnt tj = b.in[j];
    if (!(w.w < tj.thresh)) j = tj.alias_col;
    return (int32_t)j;
}

// REFILL: a lane whose path ends takes the next unassigned path of the item
// (ballot per event); otherwise each lane runs the fixed paths lane, lane + 32,
// ... of the item with no per-event bookkeeping (the autotuner picks one).
template <bool WEIGHTED, bool COUNT, bool REFILL>
__global__ void __launch_bounds__(WALK_THREADS, 5) k_batch_walk(const __grid_constant__ WalkParams a,
                                                               const __grid_constant__ BatchArgs b) {
    const int lane = threadIdx.x & 31;
    const unsigned lt_mask = (1u << lane) - 1u;
    if (*b.bad) return;
    unsigned long long paths_done = 0, jumps_done = 0;
    for (;;) {
        unsigned int item = 0;
        if (lane == 0) item = atomicAdd(b.next_item, 1u);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= b.n_items) break;
        const BatchItem it = b.items[item];
        const BatchPT p = b.pts[it.pt];
        const uint64_t p_begin = (uint64_t)it.chunk * b.chunk_len;
        const uint32_t len = (uint32_t)min((uint64_t)b.chunk_len, p.paths - p_begin);
        const uint64_t base = p.path_base + p_begin;
        const double V = b.V[p.problem];
        const float t0 = (float)p.t;
        uint32_t next = 32;
        uint32_t q = (uint32_t)lane;
        bool active = q < len;
        Walker<false> w;
        auto start_path = [&]() {
            const int32_t i0 = batch_start(b, p, a, base + q);
            w.rec = load_node(a.node, i0);
            w.j = i0; w.r = t0; w.acc = 0.0f; w.k = 0;
            w.delta = w.rec.delta;
        };
        uint32_t jumps = 0;
        auto deposit = [&]() {
            jumps += w.k;
            const int64_t slot = p.dep + (w.j - p.off);
            if (COUNT) {
                atomicAdd(b.count + slot, 1ull);
            } else {
                const double y = V * exp((double)w.acc);
                atomicAdd(b.sum1 + slot, y);
                atomicAdd(b.sum2 + slot, y * y);
            }
        };
        if (!REFILL) {
            for (; q < len; q += 32) {
                start_path();
                while (!advance<MCX_EXACT, WEIGHTED, false>(w, a, 0xFFFFFFFEu, base + q, nullptr, -1)) {
                }
                deposit();
            }
            paths_done += len;
            jumps_done += jumps;
            continue;
        }
        if (active) start_path();
        while (__any_sync(0xffffffffu, active)) {
            bool fin = false;
            if (active && advance<MCX_EXACT, WEIGHTED, false>(w, a, 0xFFFFFFFEu, base + q, nullptr, -1)) {
                fin = true;
                deposit();
            }
            const unsigned fm = __ballot_sync(0xffffffffu, fin);
            if (fm) {
                if (fin) {
                    q = next + (uint32_t)__popc(fm & lt_mask);
                    active = q < len;
                    if (active) start_path();
                }
                next += (uint32_t)__popc(fm);
            }
        }
        paths_done += len;
        jumps_done += jumps;
    }
#pragma unroll
    for (int sh = 16; sh > 0; sh >>= 1) jumps_done += __shfl_xor_sync(0xffffffffu, jumps_done, sh);
    if (lane == 0 && paths_done) {
        unsigned long long *ctr = reinterpret_cast<unsigned long long *>(a.status + 2);
        atomicAdd(ctr, paths_done);
        atomicAdd(ctr + 1, jumps_done);
    }
}

// One block per (problem, time): x = V c / M (or sum1 / M) and the standard error.
__global__ void k_batch_finish(const BatchPT *__restrict__ pts, BatchArgs b, double *x, double *sem,
                               uint32_t *status) {
    const BatchPT p = pts[blockIdx.x];
    const double M = (double)p.paths;
    const double V = b.V[p.problem];
    for (int64_t i = threadIdx.x; i < p.n; i += blockDim.x) {
        const int64_t s = p.dep + i;
        if (*b.bad) {
            x[s] = QNAN;
            sem[s] = QNAN;
            continue;
        }
        double s1, s2;
        if (b.count) {
            const double c = (double)b.count[s];
            s1 = V * c;
            s2 = V * V * c;
        } else {
            s1 = b.sum1[s];
            s2 = b.sum2[s];
        }
        const double mu = s1 / M;
        double var = M > 1.0 ? (s2 - s1 * mu) / (M - 1.0) : 0.0;
        if (var < 0.0) var = 0.0;
        x[s] = mu;
        sem[s] = sqrt(var / M);
        if (!isfinite(mu) || !isfinite(var)) atomicOr(status, ST_OVERFLOW);
    }
    if (*b.bad && blockIdx.x == 0 && threadIdx.x == 0) atomicOr(status, ST_BAD_V);
}

}  // namespace
}  // namespace mcx

using namespace mcx;

struct mcx_batch {
    int32_t problems = 0;
    int32_t n_pt = 0;
    int64_t N = 0;          // padded states
    int64_t ngroups = 0;
    int64_t slots = 0;      // sum over pairs of n_b
    uint64_t total_paths = 0;
    mcx_plan *plan = nullptr;
    std::vector<BatchPT> pt_host;
    std::vector<double> cost_per_path;  // per pair
    BatchPT *pts = nullptr;
    BatchPT *pbase = nullptr;  // per problem (first pair of each problem)
    int32_t *gprob = nullptr;
    double *v = nullptr;
    double *S = nullptr;
    AliasEnt *top = nullptr, *in = nullptr;
    double *q = nullptr;
    int32_t *stack = nullptr;
    double *V = nullptr;
    uint32_t *bad = nullptr;
    unsigned int *next_item = nullptr;
    void *dep = nullptr;
    double *x = nullptr, *sem = nullptr;
    BatchItem *items = nullptr;
    uint32_t n_items = 0;
    uint32_t chunk = 0;
    int blocks_per_sm = 0;
    bool refill = true;  // lane refill (autotuned)
    int sms = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphNode_t walk_node = nullptr;
    WalkParams wp{};
    BatchArgs ba{};
    bool count_mode = true;
    double tuned_ms = 0.0;
};

namespace {

mcx_status st_from(cudaError_t e) {
    if (e == cudaSuccess) return MCX_OK;
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return MCX_E_OOM;
    }
    return MCX_E_CUDA;
}

void free_batch(mcx_batch *b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    void *bufs[] = {b->pts, b->pbase, b->gprob, b->v, b->S, b->top, b->in, b->q, b->stack, b->V, b->bad,
                    b->next_item, b->dep, b->x, b->sem, b->items};
    for (void *p : bufs) dev_free(p);
    if (b->plan) mcx_plan_destroy(b->plan);
    delete b;
}

template <bool REFILL>
void *walk_func_r(bool weighted, bool count) {
    if (weighted) return count ? (void *)k_batch_walk<true, true, REFILL> : (void *)k_batch_walk<true, false, REFILL>;
    return count ? (void *)k_batch_walk<false, true, REFILL> : (void *)k_batch_walk<false, false, REFILL>;
}

void *walk_func(bool weighted, bool count, bool refill) {
    return refill ? walk_func_r<true>(weighted, count) : walk_func_r<false>(weighted, count);
}

template <bool REFILL>
void launch_walk(const mcx_batch *b, bool weighted, unsigned grid, cudaStream_t cs);

// Work items for chunk length L, largest estimated item cost first; with
// stride > 1 only every stride-th item is kept (the autotuner's sample).
cudaError_t make_items(mcx_batch *b, uint32_t L, cudaStream_t st, uint32_t stride = 1) {
    std::vector<int32_t> order(b->n_pt);
    for (int32_t i = 0; i < b->n_pt; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(),
                     [b](int32_t x, int32_t y) { return b->cost_per_path[x] > b->cost_per_path[y]; });
    std::vector<BatchItem> items;
    uint64_t idx = 0;
    for (int32_t k : order) {
        const uint64_t chunks = (b->pt_host[k].paths + L - 1) / L;
        for (uint64_t c = 0; c < chunks; ++c, ++idx)
            if (idx % stride == 0) items.push_back(BatchItem{(uint32_t)k, (uint32_t)c});
    }
    dev_free(b->items);
    b->items = nullptr;
    cudaError_t e = dev_malloc(&b->items, sizeof(BatchItem) * (items.size() + 1));
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(b->items, items.data(), sizeof(BatchItem) * items.size(), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    e = cudaStreamSynchronize(st);
    b->n_items = (uint32_t)items.size();
    b->chunk = L;
    return e;
}

// Capture reset + walk + finish into a graph for the current schedule.
template <bool REFILL>
void launch_walk(const mcx_batch *b, bool weighted, unsigned grid, cudaStream_t cs) {
    if (weighted) {
        if (b->count_mode) k_batch_walk<true, true, REFILL><<<grid, WALK_THREADS, 0, cs>>>(b->wp, b->ba);
        else k_batch_walk<true, false, REFILL><<<grid, WALK_THREADS, 0, cs>>>(b->wp, b->ba);
    } else {
        if (b->count_mode) k_batch_walk<false, true, REFILL><<<grid, WALK_THREADS, 0, cs>>>(b->wp, b->ba);
        else k_batch_walk<false, false, REFILL><<<grid, WALK_THREADS, 0, cs>>>(b->wp, b->ba);
    }
}

// The start tables of every problem from the batch's current v (Lemma 2: j ~ v/V):
// group sums, per-problem top tables, member tables (one warp per group); an
// invalid v anywhere latches `bad` (the walk then does nothing and the finish
// writes NaN).  Enqueued at creation and inside every run's graph, so new
// values (mcx_batch_set_v) take effect at the next run.
cudaError_t enqueue_tables(mcx_batch *b, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(b->bad, 0, 16, st);
    if (e != cudaSuccess) return e;
    const unsigned gb = (unsigned)((b->ngroups + 127) / 128);
    k_bgroup_sums<<<gb, 128, 0, st>>>(b->ngroups, b->gprob, b->pbase, b->v, b->S, b->bad);
    k_btop<<<(b->problems + 63) / 64, 64, 0, st>>>(b->problems, b->pbase, b->S, b->top, b->q, b->stack, b->V, b->bad);
    k_binner<<<(unsigned)((b->ngroups + 3) / 4), 128, 0, st>>>(b->ngroups, b->gprob, b->pbase, b->v, b->S, b->in, b->q,
                                                              b->stack);
    return cudaGetLastError();
}

cudaError_t capture(mcx_batch *b, cudaStream_t st) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    b->ba.items = b->items;
    b->ba.n_items = b->n_items;
    b->ba.chunk_len = b->chunk;
    const bool weighted = b->plan->weighted_rows > 0;
    cudaStream_t cs;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaMemsetAsync(b->next_item, 0, sizeof(unsigned int), cs);
        cudaMemsetAsync(b->dep, 0, (b->count_mode ? 8 : 16) * (size_t)b->slots, cs);
        enqueue_tables(b, cs);
        const unsigned grid = (unsigned)(b->sms * b->blocks_per_sm);
        if (b->refill) launch_walk<true>(b, weighted, grid, cs);
        else launch_walk<false>(b, weighted, grid, cs);
        k_batch_finish<<<b->n_pt, 256, 0, cs>>>(b->pts, b->ba, b->x, b->sem, b->plan->status);
        e = cudaStreamEndCapture(cs, &b->graph);
    }
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) return e;
    e = cudaGraphInstantiate(&b->exec, b->graph, 0);
    if (e != cudaSuccess) return e;
    // find the walk node (its seed is updated per run)
    size_t nn = 0;
    cudaGraphGetNodes(b->graph, nullptr, &nn);
    std::vector<cudaGraphNode_t> nodes(nn);
    cudaGraphGetNodes(b->graph, nodes.data(), &nn);
    const void *wf = walk_func(weighted, b->count_mode, b->refill);
    for (auto nd : nodes) {
        cudaGraphNodeType ty;
        cudaGraphNodeGetType(nd, &ty);
        if (ty != cudaGraphNodeTypeKernel) continue;
        cudaKernelNodeParams kp;
        if (cudaGraphKernelNodeGetParams(nd, &kp) == cudaSuccess && kp.func == wf) b->walk_node = nd;
    }
    return b->walk_node ? cudaSuccess : cudaErrorUnknown;
}

cudaError_t run_graph(mcx_batch *b, uint64_t seed, cudaStream_t st) {
    set_round_keys(b->wp, seed);
    void *args[] = {&b->wp, &b->ba};
    cudaKernelNodeParams kp;
    cudaError_t e = cudaGraphKernelNodeGetParams(b->walk_node, &kp);
    if (e != cudaSuccess) return e;
    kp.kernelParams = args;
    kp.extra = nullptr;
    e = cudaGraphExecKernelNodeSetParams(b->exec, b->walk_node, &kp);
    if (e != cudaSuccess) return e;
    return cudaGraphLaunch(b->exec, st);
}

std::string signature(const mcx_batch *b) {
    char buf[512];
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp pr;
    cudaGetDeviceProperties(&pr, dev);
    snprintf(buf, sizeof buf, "%s|pairs=%d|states=%lld|paths=%llu|nnz=%lld|w=%d", pr.name, b->n_pt,
             (long long)b->N, (unsigned long long)b->total_paths, (long long)b->plan->nnz_off,
             b->plan->weighted_rows > 0 ? 1 : 0);
    return buf;
}

// Cached schedule of a problem-set signature: chunk, blocks per SM, lane refill
// ("refill" 1 when absent).
bool cache_lookup(const char *path, const std::string &key, uint32_t *L, int *bps, bool *refill) {
    long c = 0, k = 0, r = 1;
    if (!tune_cache_get(path, key, "chunk", &c) || !tune_cache_get(path, key, "blocks_per_sm", &k)) return false;
    tune_cache_get(path, key, "refill", &r);
    *L = (uint32_t)c;
    *bps = (int)k;
    *refill = r != 0;
    return c > 0 && k > 0;
}

void cache_store(const char *path, const std::string &key, uint32_t L, int bps, bool refill, double ms) {
    tune_cache_put(path, key, {{"chunk", (long)L}, {"blocks_per_sm", (long)bps}, {"refill", refill ? 1L : 0L}}, ms);
}

}  // namespace

extern "C" {

mcx_status mcx_batch_create(int32_t count, const mcx_problem *pr, const char *tune_cache, void *stream,
                            mcx_batch **out) {
    NvtxRange nvtx("mcx_batch_create");
    if (!out) return MCX_E_INVALID;
    *out = nullptr;
    if (count < 1 || !pr) return MCX_E_INVALID;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    mcx_batch *b = new (std::nothrow) mcx_batch();
    if (!b) return MCX_E_OOM;
    b->problems = count;
    // layout and validation of the host descriptions
    std::vector<int64_t> off(count);
    int64_t N = 0, nnz = 0;
    for (int32_t i = 0; i < count; ++i) {
        const mcx_problem &p = pr[i];
        if (p.n < 1 || p.nnz < 0 || !p.row_ptr || (p.nnz > 0 && (!p.col || !p.val)) || !p.v || p.n_times < 1 ||
            !p.times || p.paths < 1 || p.paths > (1ull << 40)) {
            delete b;
            return MCX_E_INVALID;
        }
        if (p.row_ptr[0] != 0 || p.row_ptr[p.n] != p.nnz) {
            delete b;
            return MCX_E_INVALID;
        }
        for (int32_t k = 0; k < p.n_times; ++k)
            if (!(p.times[k] > 0.0) || !isfinite(p.times[k])) {
                delete b;
                return MCX_E_INVALID;
            }
        off[i] = N;
        N += (p.n + BGROUP - 1) / BGROUP * BGROUP;
        nnz += p.nnz;
    }
    if (N >= (int64_t)0x7fffffff) {
        delete b;
        return MCX_E_INVALID;
    }
    b->N = N;
    b->ngroups = N / BGROUP;
    // block-diagonal CSR on the host (columns shifted by the block offset)
    std::vector<int64_t> rp(N + 1, 0);
    std::vector<int32_t> col((size_t)std::max<int64_t>(nnz, 1));
    std::vector<double> val((size_t)std::max<int64_t>(nnz, 1));
    std::vector<double> v((size_t)N, 0.0);
    std::vector<int32_t> gprob((size_t)b->ngroups, -1);
    int64_t w = 0;
    for (int32_t i = 0; i < count; ++i) {
        const mcx_problem &p = pr[i];
        for (int64_t r = 0; r < p.n; ++r) {
            rp[off[i] + r] = w;
            for (int64_t q = p.row_ptr[r]; q < p.row_ptr[r + 1]; ++q) {
                if (p.col[q] < 0 || p.col[q] >= p.n) {
                    delete b;
                    return MCX_E_INVALID;
                }
                col[w] = (int32_t)(p.col[q] + off[i]);
                val[w] = p.val[q];
                ++w;
            }
            v[off[i] + r] = p.v[r];
        }
        const int64_t end = (i + 1 < count) ? off[i + 1] : N;
        for (int64_t r = off[i] + p.n; r < end; ++r) rp[r] = w;
        for (int64_t g = off[i] / BGROUP; g < (off[i] + p.n + BGROUP - 1) / BGROUP; ++g) gprob[g] = i;
    }
    rp[N] = w;
    mcx_status rc = mcx_plan_create(N, w, rp.data(), col.data(), val.data(), MCX_PLAN_HOST_INPUT, stream, &b->plan);
    if (rc != MCX_OK) {
        free_batch(b);
        return rc;
    }
    // (problem, time) pairs
    int64_t slots = 0;
    for (int32_t i = 0; i < count; ++i) {
        const mcx_problem &p = pr[i];
        double lam = 0.0;  // mean jump rate for the cost model
        for (int64_t r = 0; r < p.n; ++r)
            for (int64_t q = p.row_ptr[r]; q < p.row_ptr[r + 1]; ++q)
                if (p.col[q] != r && p.val[q] > 0.0) lam += p.val[q];
        lam /= (double)p.n;
        for (int32_t k = 0; k < p.n_times; ++k) {
            BatchPT t{};
            t.off = off[i];
            t.n = p.n;
            t.g0 = off[i] / BGROUP;
            t.G = (p.n + BGROUP - 1) / BGROUP;
            t.paths = p.paths;
            t.path_base = (uint64_t)b->pt_host.size() << 40;
            t.dep = slots;
            t.problem = i;
            t.tidx = k;
            t.t = p.times[k];
            slots += p.n;
            b->total_paths += p.paths;
            b->pt_host.push_back(t);
            b->cost_per_path.push_back(1.0 + p.times[k] * lam);
        }
    }
    b->n_pt = (int32_t)b->pt_host.size();
    b->slots = slots;
    b->count_mode = b->plan->zero_potential;
    std::vector<BatchPT> pbase(count);
    for (const auto &t : b->pt_host)
        if (t.tidx == 0) pbase[t.problem] = t;
    cudaError_t e = cudaSuccess;
    const int64_t m = std::max<int64_t>(N, b->ngroups);
    do {
        if ((e = dev_malloc(&b->pts, sizeof(BatchPT) * b->n_pt)) != cudaSuccess) break;
        if ((e = dev_malloc(&b->pbase, sizeof(BatchPT) * count)) != cudaSuccess) break;
        if ((e = dev_malloc(&b->gprob, sizeof(int32_t) * b->ngroups)) != cudaSuccess) break;
        if ((e = dev_malloc(&b->v, sizeof(double) * N)) != cudaSuccess) break;
        if ((e = dev_malloc(&b->S, sizeof(double) * b->ngroups)) != cudaSuccess) break;
        if ((e = dev_malloc(&b->top, sizeof(AliasEnt) * b->ngroups)) != cudaSuccess) break;
        if ((e = dev_malloc(&b->in, sizeof(AliasEnt) * N)) != cudaSuccess) break;
        if ((e = dev_malloc(&b->q, sizeof(double) * m)) != cudaSuccess) break;
        if ((e = dev_malloc(&b->stack, sizeof(int32_t) * m)) != cudaSuccess) break;
        if ((e = dev_malloc(&b->V, sizeof(double) * count)) != cudaSuccess) break;
        if ((e = dev_malloc(&b->bad, 16)) != cudaSuccess) break;
        if ((e = dev_malloc(&b->next_item, 16)) != cudaSuccess) break;
        if ((e = dev_malloc(&b->dep, (b->count_mode ? 8 : 16) * (size_t)slots)) != cudaSuccess) break;
        if ((e = dev_malloc(&b->x, sizeof(double) * slots)) != cudaSuccess) break;
        if ((e = dev_malloc(&b->sem, sizeof(double) * slots)) != cudaSuccess) break;
        cudaMemcpyAsync(b->pts, b->pt_host.data(), sizeof(BatchPT) * b->n_pt, cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(b->pbase, pbase.data(), sizeof(BatchPT) * count, cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(b->gprob, gprob.data(), sizeof(int32_t) * b->ngroups, cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(b->v, v.data(), sizeof(double) * N, cudaMemcpyHostToDevice, st);
        if ((e = enqueue_tables(b, st)) != cudaSuccess) break;
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) break;
        uint32_t hbad = 0;
        cudaMemcpy(&hbad, b->bad, 4, cudaMemcpyDeviceToHost);
        if (hbad) {
            free_batch(b);
            return MCX_E_NEG_V;
        }
        // walker parameters (EXACT functional, FP32 paths)
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
        BatchArgs &ba = b->ba;
        ba.pts = b->pts;
        ba.next_item = b->next_item;
        ba.top = b->top;
        ba.in = b->in;
        ba.V = b->V;
        ba.bad = b->bad;
        if (b->count_mode) {
            ba.count = static_cast<unsigned long long *>(b->dep);
        } else {
            ba.sum1 = static_cast<double *>(b->dep);
            ba.sum2 = static_cast<double *>(b->dep) + slots;
        }
        // schedule: cached, else autotuned over lane refill x chunk x blocks-per-SM (one timed run each)
        const std::string key = signature(b);
        uint32_t L = 0;
        int bps = 0;
        bool rf = true;
        if (cache_lookup(tune_cache, key, &L, &bps, &rf)) {
            b->blocks_per_sm = bps;
            b->refill = rf;
            if ((e = make_items(b, L, st)) != cudaSuccess) break;
            if ((e = capture(b, st)) != cudaSuccess) break;
        } else {
            const uint32_t Ls[] = {512, 1024, 2048, 4096};
            const int bpss[] = {2, 3, 4, 5};  // 49 registers: at most 5 resident blocks of 256
            // lane refill on over the (chunk, blocks per SM) grid, then refill off at
            // the best of those; refill off is kept only if it wins the sample by more
            // than 5% (a closer win did not carry over to the full batch)
            double best_r[2] = {1e300, 1e300};
            uint32_t bestL_r[2] = {4096, 4096};
            int bestb_r[2] = {4, 4};
            cudaEvent_t e0, e1;
            cudaEventCreate(&e0);
            cudaEventCreate(&e1);
            auto time_setting = [&](uint32_t Lc, int bc, int rc) -> cudaError_t {
                b->refill = rc != 0;
                b->blocks_per_sm = bc;
                cudaError_t er;
                if ((er = capture(b, st)) != cudaSuccess) return er;
                if ((er = run_graph(b, 0x5eed, st)) != cudaSuccess) return er;  // warm
                cudaEventRecord(e0, st);
                if ((er = run_graph(b, 0x5eed, st)) != cudaSuccess) return er;
                cudaEventRecord(e1, st);
                if ((er = cudaEventSynchronize(e1)) != cudaSuccess) return er;
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (ms < best_r[rc]) {
                    best_r[rc] = ms;
                    bestL_r[rc] = Lc;
                    bestb_r[rc] = bc;
                }
                return cudaSuccess;
            };
            for (uint32_t Lc : Ls) {
                // time each setting on every 8th work item of the cost-ordered list
                if ((e = make_items(b, Lc, st, 8)) != cudaSuccess) break;
                for (int bc : bpss)
                    if ((e = time_setting(Lc, bc, 1)) != cudaSuccess) break;
                if (e != cudaSuccess) break;
            }
            if (e == cudaSuccess && (e = make_items(b, bestL_r[1], st, 8)) == cudaSuccess)
                e = time_setting(bestL_r[1], bestb_r[1], 0);
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            if (e != cudaSuccess) break;
            const int pick = best_r[0] < 0.95 * best_r[1] ? 0 : 1;
            const double best = best_r[pick];
            const uint32_t bestL = bestL_r[pick];
            const int bestb = bestb_r[pick];
            const bool bestr = pick == 1;
            b->blocks_per_sm = bestb;
            b->refill = bestr;
            b->tuned_ms = best;
            if ((e = make_items(b, bestL, st)) != cudaSuccess) break;
            if ((e = capture(b, st)) != cudaSuccess) break;
            cache_store(tune_cache, key, bestL, bestb, bestr, best);
        }
        // clear the tuning runs' statistics
        cudaMemsetAsync(b->plan->status, 0, 32, st);
        e = cudaStreamSynchronize(st);
    } while (0);
    if (e != cudaSuccess) {
        free_batch(b);
        return st_from(e);
    }
    *out = b;
    return MCX_OK;
}

mcx_status mcx_batch_run(mcx_batch *b, uint64_t seed, void *stream) {
    NvtxRange nvtx("mcx_batch_run");
    if (!b) return MCX_E_INVALID;
    return st_from(run_graph(b, seed, static_cast<cudaStream_t>(stream)));
}

mcx_status mcx_batch_set_v(mcx_batch *b, int32_t problem, const double *v, void *stream) {
    NvtxRange nvtx("mcx_batch_set_v");
    if (!b || problem < 0 || problem >= b->problems || !v) return MCX_E_INVALID;
    for (const auto &t : b->pt_host) {
        if (t.problem != problem) continue;
        return st_from(cudaMemcpyAsync(b->v + t.off, v, sizeof(double) * (size_t)t.n, cudaMemcpyDeviceToDevice,
                                       static_cast<cudaStream_t>(stream)));
    }
    return MCX_E_INVALID;
}

mcx_status mcx_batch_result(const mcx_batch *b, int32_t problem, int32_t time_index, double *x, double *sem,
                            void *stream) {
    if (!b || problem < 0 || problem >= b->problems || !x) return MCX_E_INVALID;
    for (const auto &t : b->pt_host) {
        if (t.problem != problem || t.tidx != time_index) continue;
        cudaStream_t st = static_cast<cudaStream_t>(stream);
        cudaError_t e = cudaMemcpyAsync(x, b->x + t.dep, sizeof(double) * t.n, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess && sem)
            e = cudaMemcpyAsync(sem, b->sem + t.dep, sizeof(double) * t.n, cudaMemcpyDeviceToDevice, st);
        return st_from(e);
    }
    return MCX_E_INVALID;
}

mcx_status mcx_batch_get_info(const mcx_batch *b, mcx_batch_info *info) {
    if (!b || !info) return MCX_E_INVALID;
    info->problems = b->problems;
    info->pairs = b->n_pt;
    info->states = b->N;
    info->total_paths = b->total_paths;
    info->work_items = b->n_items;
    info->chunk = b->chunk;
    info->blocks_per_sm = b->blocks_per_sm;
    info->grid = b->sms * b->blocks_per_sm;
    info->lane_refill = b->refill ? 1 : 0;
    info->count_deposits = b->count_mode ? 1 : 0;
    info->tuned_ms = b->tuned_ms;
    return MCX_OK;
}

mcx_status mcx_batch_sync(mcx_batch *b, void *stream, mcx_stats *stats) {
    if (!b) return MCX_E_INVALID;
    return mcx_sync(b->plan, stream, stats);
}

void mcx_batch_destroy(mcx_batch *b) {
    if (!b) return;
    cudaDeviceSynchronize();
    free_batch(b);
}

}  // extern "C"
