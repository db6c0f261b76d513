// Problem preparation: the decomposition A = D - L of Sec. 2 and the O(1)
// jump tables of Sec. 4.
//
//   k_prep_rows   validates each CSR row and computes, in CSR order and FP64,
//                 lambda_i = sum_{j != i, a_ij > 0} a_ij, delta_i = a_ii + lambda_i,
//                 the kept-entry count deg_i and whether the row is uniform
//                 (all kept values bit-equal: jumps pick a slot uniformly,
//                 Sec. 4) or weighted (jumps need an alias table).
//   k_scan_*      exclusive prefix sum of deg -> row_start (int64), plus the
//                 totals (kept entries, max degree, weighted rows).
//   k_prep_fill   copies the kept columns and builds, for weighted rows, the
//                 canonical Vose alias table: scaled weights q_k = (a_k d)/lambda,
//                 "small" (q < 1) and "large" index lists in index order, pairs
//                 popped from the back, the large entry keeps (q_l + q_s) - 1,
//                 leftovers alias themselves; the kept-own-column probability is
//                 stored as floor(q 2^32).
//
// Rows are handled one per thread with sequential FP64 sums, so every value
// is independent of the launch shape.  Preparation is O(nnz) streaming work,
// run once per matrix.
#include <math.h>

#include "mcx_internal.cuh"
#include "launch.h"

namespace mcx {
namespace {

constexpr int PREP_THREADS = 256;
constexpr int SCAN_THREADS = 1024;
constexpr int SCAN_ITEMS = 2;  // rows per thread in a scan tile
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

struct PrepTotals {
    unsigned long long nnz_off;
    unsigned long long weighted_rows;
    int max_deg;
    uint32_t status;
    uint32_t nonzero_potential;
    uint32_t pad;
};

__global__ void k_prep_rows(int64_t n, int64_t nnz, const int64_t *__restrict__ row_ptr,
                            const int32_t *__restrict__ col, const double *__restrict__ val,
                            NodeRec *__restrict__ node, NodeRec64 *__restrict__ node64, int32_t *__restrict__ deg_out,
                            PrepTotals *tot) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0 && (row_ptr[0] != 0 || row_ptr[n] != nnz)) atomicOr(&tot->status, ST_BAD_STRUCT);
    if (i >= n) return;
    const int64_t p0 = row_ptr[i];
    const int64_t p1 = row_ptr[i + 1];
    uint32_t bad = 0;
    int32_t d = 0;
    double lam = 0.0, diag = 0.0;
    bool uniform = true;
    unsigned long long first_bits = 0;
    if (p0 < 0 || p1 < p0 || p1 > nnz) {
        bad |= ST_BAD_STRUCT;
    } else {
        int32_t prev = -1;
        for (int64_t p = p0; p < p1; ++p) {
            const int32_t c = col[p];
            const double a = val[p];
            if (c < 0 || c >= n || c <= prev) {
                bad |= ST_BAD_STRUCT;
                break;
            }
            prev = c;
            if (!isfinite(a)) {
                bad |= ST_NONFINITE;
                continue;
            }
            if (c == i) {
                diag = a;
            } else if (a < 0.0) {
                bad |= ST_NEG_OFFDIAG;
            } else if (a > 0.0) {
                const unsigned long long bits = (unsigned long long)__double_as_longlong(a);
                if (d == 0) first_bits = bits;
                else if (bits != first_bits) uniform = false;
                lam = __dadd_rn(lam, a);
                ++d;
            }
        }
    }
    const double delta = __dadd_rn(diag, lam);
    const double inv = d > 0 ? __ddiv_rn(1.0, lam) : 0.0;
    // a rate whose FP32 reciprocal is 0 (or an infinite rate/potential) would give
    // zero holding times and a path that never ends: reject it
    if (!bad && (!isfinite(lam) || !isfinite(delta) || (d > 0 && __double2float_rn(inv) == 0.0f) ||
                 !isfinite(__double2float_rn(delta))))
        bad |= ST_NONFINITE;
    if (bad) {
        atomicOr(&tot->status, bad);
        d = 0;
    }
    deg_out[i] = d;
    if (delta != 0.0) atomicOr(&tot->nonzero_potential, 1u);
    NodeRec r;
    r.row_start = 0;  // filled by the scan
    r.deg = d;
    r.flags = (d > 1 && !uniform) ? NODE_WEIGHTED : 0u;
    r.inv_rate = __double2float_rn(inv);
    r.delta = __double2float_rn(delta);
    r.v = 0.0f;
    r.pad = 0u;
    node[i] = r;
    node64[i] = NodeRec64{inv, delta, 0.0, 0.0};
}

// Tile scan: exclusive prefix of deg within each SCAN_TILE rows; tile totals to tile_sum.
__global__ void k_scan_tiles(int64_t n, const int32_t *__restrict__ deg, int64_t *__restrict__ excl,
                             int64_t *__restrict__ tile_sum, PrepTotals *tot, const NodeRec *__restrict__ node) {
    __shared__ int64_t warp_tot[SCAN_THREADS / 32];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    int64_t v[SCAN_ITEMS];
    int64_t local = 0;
    int my_max = 0;
    unsigned long long my_weighted = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        const int64_t i = base + k;
        const int32_t d = i < n ? deg[i] : 0;
        v[k] = local;
        local += d;
        my_max = max(my_max, d);
        if (i < n && (node[i].flags & NODE_WEIGHTED)) ++my_weighted;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t incl = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int64_t w = lane < SCAN_THREADS / 32 ? warp_tot[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < SCAN_THREADS / 32) warp_tot[lane] = w;  // inclusive over warps
    }
    __syncthreads();
    const int64_t warp_off = warp > 0 ? warp_tot[warp - 1] : 0;
    const int64_t thread_off = warp_off + incl - local;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        const int64_t i = base + k;
        if (i < n) excl[i] = thread_off + v[k];
    }
    if (threadIdx.x == SCAN_THREADS - 1) tile_sum[blockIdx.x] = thread_off + local;
    // totals
    for (int o = 16; o > 0; o >>= 1) {
        my_max = max(my_max, __shfl_xor_sync(0xffffffffu, my_max, o));
        my_weighted += __shfl_xor_sync(0xffffffffu, my_weighted, o);
    }
    if (lane == 0) {
        atomicMax(&tot->max_deg, my_max);
        if (my_weighted) atomicAdd(&tot->weighted_rows, my_weighted);
    }
}

// Exclusive scan of the tile totals by one block (sequential over chunks of 1024).
__global__ void k_scan_tile_sums(int64_t ntiles, int64_t *__restrict__ tile_sum, PrepTotals *tot) {
    __shared__ int64_t warp_tot[32];
    __shared__ int64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t base = 0; base < ntiles; base += blockDim.x) {
        const int64_t i = base + threadIdx.x;
        const int64_t x = i < ntiles ? tile_sum[i] : 0;
        int64_t incl = x;
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) warp_tot[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            int64_t w = lane < (int)(blockDim.x / 32) ? warp_tot[lane] : 0;
            for (int o = 1; o < 32; o <<= 1) {
                const int64_t y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += y;
            }
            warp_tot[lane] = w;
        }
        __syncthreads();
        const int64_t off = carry + (warp > 0 ? warp_tot[warp - 1] : 0) + incl - x;
        if (i < ntiles) tile_sum[i] = off;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = off + x;
        __syncthreads();
    }
    if (threadIdx.x == 0) tot->nnz_off = (unsigned long long)carry;
}

__global__ void k_scan_add(int64_t n, const int64_t *__restrict__ excl, const int64_t *__restrict__ tile_off,
                           NodeRec *__restrict__ node) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    node[i].row_start = excl[i] + tile_off[i / SCAN_TILE];
}

__global__ void k_prep_fill(int64_t n, const int64_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                            const double *__restrict__ val, const NodeRec *__restrict__ node,
                            int32_t *__restrict__ edge_col, AliasEnt *__restrict__ alias, double *__restrict__ qbuf,
                            int32_t *__restrict__ stack) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const NodeRec r = node[i];
    const int64_t o = r.row_start;
    const int32_t d = r.deg;
    if (d == 0) return;
    double lam = 0.0;
    int32_t k = 0;
    for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) {
        const int32_t c = col[p];
        const double a = val[p];
        if (c != i && a > 0.0) {
            edge_col[o + k] = c;
            if (r.flags & NODE_WEIGHTED) qbuf[o + k] = a;
            lam = __dadd_rn(lam, a);
            ++k;
        }
    }
    if (!(r.flags & NODE_WEIGHTED)) return;
    const int32_t *cols = edge_col + o;
    vose_build(d, qbuf + o, lam, [cols](int32_t k) { return cols[k]; }, alias + o, qbuf + o, stack + o);
}

// Pack columns and alias entries into 16-byte edge records (weighted plans).
__global__ void k_pack_edges(int64_t n, const NodeRec *__restrict__ node, const int32_t *__restrict__ edge_col,
                             const AliasEnt *__restrict__ alias, Edge16 *__restrict__ e16) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const NodeRec r = node[i];
    const bool w = (r.flags & NODE_WEIGHTED) != 0;
    for (int32_t k = 0; k < r.deg; ++k) {
        const int64_t e = r.row_start + k;
        const int32_t c = edge_col[e];
        e16[e] = w ? Edge16{c, alias[e].alias_col, alias[e].thresh, 0u} : Edge16{c, c, 0xFFFFFFFFu, 0u};
    }
}

__global__ void k_export_rows(int64_t n, const NodeRec *__restrict__ node, const NodeRec64 *__restrict__ node64,
                              int32_t *deg, int64_t *row_start, uint8_t *weighted, float *ir32, float *d32,
                              double *ir64, double *d64) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const NodeRec r = node[i];
    if (deg) deg[i] = r.deg;
    if (row_start) row_start[i] = r.row_start;
    if (weighted) weighted[i] = (uint8_t)(r.flags & NODE_WEIGHTED);
    if (ir32) ir32[i] = r.inv_rate;
    if (d32) d32[i] = r.delta;
    if (ir64) ir64[i] = node64[i].inv_rate;
    if (d64) d64[i] = node64[i].delta;
}

__global__ void k_export_edges(int64_t n, const NodeRec *__restrict__ node, const int32_t *__restrict__ edge_col,
                               const Edge16 *__restrict__ e16, int32_t *ecol, int32_t *acol, uint32_t *thr) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const NodeRec r = node[i];
    for (int32_t k = 0; k < r.deg; ++k) {
        const int64_t e = r.row_start + k;
        const int32_t c = edge_col[e];
        if (ecol) ecol[e] = c;
        if (acol) acol[e] = e16 ? e16[e].alias_col : c;
        if (thr) thr[e] = e16 ? e16[e].thresh : 0xFFFFFFFFu;
    }
}

}  // namespace

#define MCX_TRY(x)                          \
    do {                                    \
        cudaError_t e_ = (x);               \
        if (e_ != cudaSuccess) return e_;   \
    } while (0)

cudaError_t launch_prep(mcx_plan *plan, const int64_t *row_ptr, const int32_t *col, const double *val,
                        cudaStream_t st, uint32_t *host_status) {
    const int64_t n = plan->n;
    *host_status = 0;
    const int64_t ntiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    int32_t *deg = nullptr;
    int64_t *excl = nullptr, *tile_sum = nullptr;
    PrepTotals *tot_d = nullptr;
    double *qbuf = nullptr;
    int32_t *stack = nullptr;
    AliasEnt *alias = nullptr;
    cudaError_t err = cudaSuccess;
    auto cleanup = [&]() {  // stream-ordered frees to the library pool
        pool_free(deg, st); pool_free(excl, st); pool_free(tile_sum, st); pool_free(tot_d, st);
        pool_free(qbuf, st); pool_free(stack, st); pool_free(alias, st);
    };
    PrepTotals tot{};
    do {
        if ((err = pool_alloc(reinterpret_cast<void **>(&deg), sizeof(int32_t) * (size_t)(n + 1), st)) != cudaSuccess) break;
        if ((err = pool_alloc(reinterpret_cast<void **>(&excl), sizeof(int64_t) * (size_t)(n + 1), st)) != cudaSuccess) break;
        if ((err = pool_alloc(reinterpret_cast<void **>(&tile_sum), sizeof(int64_t) * (size_t)(ntiles + 1), st)) != cudaSuccess) break;
        if ((err = pool_alloc(reinterpret_cast<void **>(&tot_d), sizeof(PrepTotals), st)) != cudaSuccess) break;
        if ((err = cudaMemsetAsync(tot_d, 0, sizeof(PrepTotals), st)) != cudaSuccess) break;
        const int64_t nb = (n + PREP_THREADS - 1) / PREP_THREADS;
        if (n > 0) {
            k_prep_rows<<<(unsigned)nb, PREP_THREADS, 0, st>>>(n, plan->nnz, row_ptr, col, val, plan->node,
                                                              plan->node64, deg, tot_d);
            k_scan_tiles<<<(unsigned)ntiles, SCAN_THREADS, 0, st>>>(n, deg, excl, tile_sum, tot_d, plan->node);
            k_scan_tile_sums<<<1, 1024, 0, st>>>(ntiles, tile_sum, tot_d);
            k_scan_add<<<(unsigned)nb, PREP_THREADS, 0, st>>>(n, excl, tile_sum, plan->node);
        } else {
            k_scan_tile_sums<<<1, 1024, 0, st>>>(0, tile_sum, tot_d);
        }
        if ((err = cudaGetLastError()) != cudaSuccess) break;
        if ((err = cudaMemcpyAsync(&tot, tot_d, sizeof(PrepTotals), cudaMemcpyDeviceToHost, st)) != cudaSuccess) break;
        if ((err = cudaStreamSynchronize(st)) != cudaSuccess) break;
        *host_status = tot.status;
        if (tot.status) break;
        plan->nnz_off = (int64_t)tot.nnz_off;
        plan->max_deg = tot.max_deg;
        plan->weighted_rows = (int64_t)tot.weighted_rows;
        plan->zero_potential = tot.nonzero_potential == 0;
        const size_t m = (size_t)(plan->nnz_off > 0 ? plan->nnz_off : 1);
        if ((err = pool_alloc(reinterpret_cast<void **>(&plan->edge_col), sizeof(int32_t) * m, st)) != cudaSuccess) break;
        plan->device_bytes += (int64_t)(sizeof(int32_t) * m);
        if (plan->weighted_rows > 0) {
            if ((err = pool_alloc(reinterpret_cast<void **>(&alias), sizeof(AliasEnt) * m, st)) != cudaSuccess) break;
            if ((err = pool_alloc(reinterpret_cast<void **>(&plan->edge16), sizeof(Edge16) * m, st)) != cudaSuccess) break;
            plan->device_bytes += (int64_t)(sizeof(Edge16) * m);
            if ((err = pool_alloc(reinterpret_cast<void **>(&qbuf), sizeof(double) * m, st)) != cudaSuccess) break;
            if ((err = pool_alloc(reinterpret_cast<void **>(&stack), sizeof(int32_t) * m, st)) != cudaSuccess) break;
        }
        if (n > 0) {
            k_prep_fill<<<(unsigned)nb, PREP_THREADS, 0, st>>>(n, row_ptr, col, val, plan->node, plan->edge_col,
                                                              alias, qbuf, stack);
            if (plan->weighted_rows > 0)
                k_pack_edges<<<(unsigned)nb, PREP_THREADS, 0, st>>>(n, plan->node, plan->edge_col, alias,
                                                                   plan->edge16);
        }
        if ((err = cudaGetLastError()) != cudaSuccess) break;
        if ((err = cudaStreamSynchronize(st)) != cudaSuccess) break;
    } while (0);
    cleanup();
    return err;
}

cudaError_t launch_export(const mcx_plan *plan, int32_t *deg, int64_t *row_start, uint8_t *weighted, float *ir32,
                          float *d32, double *ir64, double *d64, int32_t *ecol, int32_t *acol, uint32_t *thr,
                          cudaStream_t st) {
    if (plan->n == 0) return cudaSuccess;
    const unsigned nb = (unsigned)((plan->n + PREP_THREADS - 1) / PREP_THREADS);
    k_export_rows<<<nb, PREP_THREADS, 0, st>>>(plan->n, plan->node, plan->node64, deg, row_start, weighted, ir32, d32,
                                               ir64, d64);
    if (ecol || acol || thr)
        k_export_edges<<<nb, PREP_THREADS, 0, st>>>(plan->n, plan->node, plan->edge_col, plan->edge16, ecol, acol, thr);
    return cudaGetLastError();
}

}  // namespace mcx
