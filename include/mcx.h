/*
 * mcx.h — C-ABI of the GB300 Monte Carlo exp(tA)v library.
 *
 * The library estimates x = exp(tA) v (the paper writes beta for t, Sec. 2)
 * for a sparse A in CSR form by simulating independent continuous-time
 * Markov-chain walkers over the indices of A (Sec. 3, Eq. paths) and
 * averaging the multiplicative functional of Theorem 1 (one entry, or any set
 * of entries: Algorithm 1) or Theorem 2 (the full vector from walkers started
 * at j ~ v/V: Algorithm 2).
 *
 * Decomposition (Sec. 2, A = D - L).  For row i:
 *   lambda_i = sum_{j != i} a_ij     the jump rate (L_ii; needs a_ij >= 0, j != i)
 *   delta_i  = sum_j a_ij            the potential (D_ii = a_ii + lambda_i)
 *   k_ij     = a_ij / lambda_i       the jump probabilities of Eq. paths
 * The paper's d_i denotes both lambda_i and delta_i; they coincide for 0/1
 * adjacency matrices.  A need not be symmetric for the backward calls; the
 * forward call walks the rows of the matrix the plan was built from, which
 * must be A^T (A itself when A is symmetric, as Theorem 2 assumes).
 *
 * Conventions shared by every call:
 *   - Pointers are device pointers unless a flag says otherwise; the caller
 *     owns every array it passes and allocates every output.  A plan owns the
 *     device buffers it creates and frees them in mcx_plan_destroy.
 *   - Calls are asynchronous on the CUDA stream passed as `stream`
 *     (a cudaStream_t; NULL means the legacy default stream).  Argument
 *     errors are returned at call time; errors found on the device (result
 *     overflow) are latched in the plan and returned by mcx_sync.
 *   - Nothing traps on the device and no C++ exception crosses this ABI.
 *   - Indices are 0-based; column indices are int32, row pointers int64.
 *   - Results are a deterministic function of (inputs, seed, path_offset)
 *     and of the launch configuration the library picks for the sizes given.
 *
 * Draw schedule (fixed, so that an independent implementation reproduces
 * every path bit for bit): one Philox4x32-10 call (Salmon et al., SC'11) per
 * walker event k = 0, 1, ..., key = {seed lo32, seed hi32}, counter =
 * {k, i, path lo32, path hi32} for a backward path of entry i.  The holding
 * time in state j is S = -ln(u) * inv_rate_j with u = (2^24 - (w0 >> 8)) 2^-24
 * (FP32) or u = (2^53 - ((w0 << 21) | (w1 >> 11))) 2^-53 (FP64), the
 * logarithm being the library's own (range reduction to [1/sqrt2, sqrt2] and
 * the artanh series, fused multiply-adds in a fixed order).  If S >= r (the
 * remaining time) the path stops; otherwise the slot (w2 * deg_j) >> 32 of
 * row j is taken, and for an alias-table row its own column is kept iff
 * w3 < threshold, else its alias column.
 */
#ifndef MCX_H
#define MCX_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MCX_OK = 0,
    MCX_E_INVALID = -1,      /* bad argument or malformed CSR (unsorted/duplicate/out-of-range columns) */
    MCX_E_NEG_OFFDIAG = -2,  /* a_ij < 0 for some j != i: -L is then not a generator (Sec. 2) */
    MCX_E_NONFINITE = -3,    /* NaN or Inf in A or v */
    MCX_E_NEG_V = -4,        /* forward form needs v >= 0 with a positive sum (Lemma 2) */
    MCX_E_CUDA = -5,         /* a CUDA runtime call failed */
    MCX_E_OOM = -6,          /* device allocation failed */
    MCX_E_TIMEOUT = -7,      /* a bounded device wait gave up */
    MCX_E_UNSUPPORTED = -8,  /* valid request outside what this library implements */
    MCX_E_OVERFLOW = -9      /* an estimate or its standard error overflowed FP64 */
} mcx_status;

/* The multiplicative functional carried along each path.
 *   MCX_EXACT : logW = integral_0^t delta(X_s) ds — the limit dt -> 0; unbiased for exp(tA)v.
 *   MCX_STRANG: logW = dt [delta(X_0)/2 + sum_{k=1}^{N-1} delta(X_{k dt}) + delta(X_t)/2];
 *               unbiased for the Strang product (Eq. eq_general1, Theorem 1).
 *   MCX_LIE   : logW = dt sum_{k=1}^{N} delta(X_{k dt}); unbiased for the Lie product (Eq. deff).
 * with dt = t/N, N = nsteps.  X is one continuous path in every mode, so the
 * visited indices do not depend on the mode. */
typedef enum { MCX_EXACT = 0, MCX_STRANG = 1, MCX_LIE = 2 } mcx_functional;

/* MCX_FP32: holding times, remaining time and logW in FP32 (per-path log
 *           scaling); weights accumulated with compensated FP32 sums per lane
 *           and FP64 across lanes.  v enters as an FP32 copy scaled by the
 *           power of two 2^-k, k the binary exponent of max |v_i| (exact), and
 *           results are scaled back by 2^k, so any scale of v within the FP64
 *           range gives the same relative accuracy.  The production path.
 * MCX_FP64: every per-path quantity in FP64.  The reference path version. */
typedef enum { MCX_FP32 = 0, MCX_FP64 = 1 } mcx_precision;

/* mcx_plan_create flags */
#define MCX_PLAN_HOST_INPUT 0x1u /* row_ptr, col, val are host pointers (copied to the device) */

typedef struct mcx_plan mcx_plan;

typedef struct {
    int64_t n;               /* rows */
    int64_t nnz;             /* stored entries of A */
    int64_t nnz_off;         /* kept off-diagonal entries (a_ij > 0, j != i) */
    int64_t weighted_rows;   /* rows whose kept entries are not all equal (alias-table rows) */
    int32_t max_deg;         /* max kept entries in a row */
    int32_t reserved;
    int64_t device_bytes;    /* device memory the plan holds */
} mcx_plan_info;

typedef struct {
    uint64_t paths;          /* walker paths simulated by mcx_estimate since the last mcx_sync */
    uint64_t jumps;          /* jumps taken by those paths */
    uint32_t status_bits;    /* latched device status (bit 0: overflow, bit 4: bad entry) */
    uint32_t reserved;
} mcx_stats;

/*
 * Build a plan for A (Sec. 2: A = D - L) from CSR arrays.
 *   n        rows (= columns), 0 <= n < 2^31
 *   nnz      stored entries, row_ptr[n] == nnz
 *   row_ptr  int64 [n+1], non-decreasing, row_ptr[0] = 0
 *   col      int32 [nnz], strictly increasing within each row, in [0, n)
 *   val      float64 [nnz], finite, >= 0 off the diagonal; each row's rate
 *            lambda_i and potential delta_i must be finite with a nonzero
 *            FP32 reciprocal rate (else MCX_E_NONFINITE)
 *   flags    MCX_PLAN_HOST_INPUT if the three arrays are host memory
 *   stream   CUDA stream; the call synchronises it before returning so that
 *            validation errors come back as its status
 *   out      receives the plan (NULL on error)
 * Entries with a_ij = 0 off the diagonal are dropped.  Each row keeps its
 * off-diagonal columns in CSR order plus, if its values differ, a Vose alias
 * table (built in FP64, stored as int32 alias column + uint32 threshold) so
 * that a jump costs O(1) (Sec. 4 notes the uniform-row O(1) case; the table
 * extends it to weighted rows).
 * Errors: MCX_E_INVALID, MCX_E_NEG_OFFDIAG, MCX_E_NONFINITE, MCX_E_OOM, MCX_E_CUDA.
 */
mcx_status mcx_plan_create(int64_t n, int64_t nnz, const int64_t *row_ptr, const int32_t *col,
                           const double *val, uint32_t flags, void *stream, mcx_plan **out);

/* Fill *info (host pointer) with the plan's sizes.  Errors: MCX_E_INVALID. */
mcx_status mcx_plan_get_info(const mcx_plan *plan, mcx_plan_info *info);

/*
 * Backward estimate (Theorem 1, Algorithm 1) of x_i = (exp(tA) v)_i for each
 * requested entry: the sample mean of W v_{X_t} over paths_per_entry
 * independent paths started at i, and its standard error.
 *   v                float64 [n]; any sign (Theorem 1 does not need v >= 0)
 *   t                horizon, t >= 0 and finite; t = 0 returns v exactly
 *   functional       mcx_functional; nsteps = N >= 1 for STRANG/LIE (ignored for EXACT)
 *   paths_per_entry  M >= 1 (M >= 2 for a standard error)
 *   entries          int32 [n_entries] row indices in [0, n), or NULL for all
 *                    rows (then n_entries must equal n); an index outside
 *                    [0, n) yields NaN outputs and MCX_E_INVALID at mcx_sync
 *   seed, path_offset  paths path_offset .. path_offset+M-1 of each entry are
 *                    simulated, so disjoint offsets give independent samples
 *                    that can be merged (checkpoint / sharding)
 *   precision        mcx_precision
 *   mean             float64 [n_entries] output
 *   sem              float64 [n_entries] output, or NULL: sqrt(s^2/M) with s^2
 *                    the unbiased sample variance of W v_{X_t}
 * The plan's copy of v is overwritten, so two estimates with different v on
 * one plan must not overlap in time (use one stream per plan).
 * Errors: MCX_E_INVALID, MCX_E_CUDA, MCX_E_OOM.
 */
mcx_status mcx_estimate(mcx_plan *plan, const double *v, double t, int functional, int32_t nsteps,
                        uint64_t paths_per_entry, const int32_t *entries, int64_t n_entries,
                        uint64_t seed, uint64_t path_offset, int precision, double *mean, double *sem,
                        void *stream);

/*
 * Forward estimate (Lemma 2, Theorem 2, Algorithm 2) of the full vector
 * x = exp(tA) v: total_paths walkers start at j ~ v_j / V (V = sum of v),
 * walk the rows of the matrix the plan was built from, which must be
 * B = A^T (A itself when A is symmetric), carry B's multiplicative
 * functional, and deposit V W at their end state: x_i = (1/M) sum V W 1{X_t = i}.
 *   v            float64 [n], v >= 0, finite, V > 0 (else NaN outputs and
 *                MCX_E_NEG_V at mcx_sync)
 *   t, functional, nsteps, precision, seed as in mcx_estimate; t = 0 returns v
 *   total_paths  M >= 1; paths path_offset .. path_offset+M-1
 *   x, sem       float64 [n] outputs (sem may be NULL); sem is the standard
 *                error of the per-state mean of V W 1{X_t = i}
 * The start draw is a two-level alias over v: groups of 1024 indices with
 * sums S_g (summed in index order), V = sum of the S_g (group order), a Vose
 * table over the groups and one inside each group; one Philox call with
 * counter {0, 0xFFFFFFFF, path lo32, path hi32} (words 0-1 pick the group,
 * words 2-3 the member); walk events use counter {k, 0xFFFFFFFE, path}.
 * When every potential of the plan is exactly zero (B a CTMC generator, so
 * W = 1) the deposits are exact integer counts, so sum_i x_i = V up to one
 * rounding per entry; otherwise they are FP64 atomic sums (summation order,
 * and so the last bits, vary between runs).  The plan allocates its forward
 * scratch (about 36 n bytes) on first use.
 * Errors: MCX_E_INVALID, MCX_E_CUDA, MCX_E_OOM.
 */
mcx_status mcx_estimate_forward(mcx_plan *plan, const double *v, double t, int functional, int32_t nsteps,
                                uint64_t total_paths, uint64_t seed, uint64_t path_offset, int precision,
                                double *x, double *sem, void *stream);

/*
 * Total communicability TC(t) = 1^T exp(tA) 1 = sum_ij (exp(tA))_ij (Sec. 6,
 * with t = beta) from the forward form with v = 1 (Theorem 2, Algorithm 2):
 * the same paths as mcx_estimate_forward with v = 1 (start uniform over the
 * n states through the same two-level table and draw schedule), but instead of
 * a histogram only the mean path weight is kept: TC = n E[W].  The plan must be
 * built from A^T (A itself when A is symmetric).
 *   t, functional, nsteps, precision, seed, path_offset as in mcx_estimate_forward
 *   total_paths  M >= 2
 *   tc, sem      float64 [1] device outputs: the estimate and its standard
 *                error (sem may be NULL); t = 0 gives n exactly (synchronising)
 * Per-warp partial sums of W (log-sum-exp shifted, compensated within lanes)
 * are merged in warp order, so the result is deterministic.  Uses the plan's
 * forward scratch (the start tables of v = 1 are built on the first call and
 * kept until a forward call with another v replaces them) and grows its
 * partial-sum scratch as needed.
 * Errors: MCX_E_INVALID, MCX_E_CUDA, MCX_E_OOM; MCX_E_OVERFLOW at mcx_sync.
 */
mcx_status mcx_total_communicability(mcx_plan *plan, double t, int functional, int32_t nsteps,
                                     uint64_t total_paths, uint64_t seed, uint64_t path_offset, int precision,
                                     double *tc, double *sem, void *stream);

/*
 * Per-path record of forward paths first_path .. first_path+count-1 (same
 * arguments as mcx_estimate_forward): start (int32), end (int32), njumps
 * (uint32), hash (uint64, FNV-1a over the visited indices from the start),
 * logw (float64).  Errors: MCX_E_INVALID, MCX_E_CUDA.
 */
mcx_status mcx_trace_forward(mcx_plan *plan, const double *v, double t, int functional, int32_t nsteps,
                             uint64_t seed, uint64_t first_path, uint32_t count, int precision, int32_t *start,
                             int32_t *end, uint32_t *njumps, uint64_t *hash, double *logw, void *stream);

/*
 * x ~ exp(tA) v in one call (Theorem 1, Algorithm 1, with the beta setup of
 * Sec. 6): plan creation, optionally the power iteration for lambda_max, the
 * backward estimate of the requested entries and the status check.
 *   n, nnz, row_ptr, col, val   the CSR of A, as for mcx_plan_create
 *   v                float64 [n]
 *   t                horizon; t <= 0 asks for t = beta_scale / lambda_max(A)
 *                    (power iteration to 1e-10 relative, at most 1000 steps)
 *   beta_scale       used only when t <= 0 (beta = 1/lambda_max: 1)
 *   functional, nsteps, paths_per_entry, entries, n_entries, seed,
 *   path_offset, precision    as for mcx_estimate
 *   flags            MCX_PLAN_HOST_INPUT: every array argument (row_ptr, col,
 *                    val, v, entries, mean, sem) is host memory; the call
 *                    copies the inputs to the device and the results back
 *                    (page-locked host memory makes the copies asynchronous
 *                    DMA); 0: every array is device memory
 *   mean, sem        float64 [n_entries] outputs (sem may be NULL)
 *   t_used           host double, may be NULL: the horizon that was used
 * Device temporaries come from the library's memory pool and are returned to
 * it; the call synchronises `stream` and returns the plan's device status.
 * Errors: those of mcx_plan_create, mcx_power_iteration, mcx_estimate and
 * mcx_sync.
 */
mcx_status mcx_expm_multiply(int64_t n, int64_t nnz, const int64_t *row_ptr, const int32_t *col, const double *val,
                             const double *v, double t, double beta_scale, int functional, int32_t nsteps,
                             uint64_t paths_per_entry, const int32_t *entries, int64_t n_entries, uint64_t seed,
                             uint64_t path_offset, int precision, uint32_t flags, double *mean, double *sem,
                             double *t_used, void *stream);

/*
 * mcx_estimate without any device allocation.  The paper has no counterpart:
 * this exists for callers that cannot call cudaMalloc once they are running,
 * e.g. a service that reserves all of its device memory at start-up and must
 * keep its footprint fixed afterwards, or a host framework whose own pool
 * allocator owns the device memory and forbids outside allocations.
 * mcx_estimate may grow plan scratch with cudaMalloc (and cudaFree the old
 * block, which can synchronise the device); this call never does.
 *
 * Arguments, outputs and results are those of mcx_estimate (same kernels,
 * same chunking, same numbers).  The per-chunk partial sums live in a
 * fixed device array compiled into the library, of 131072 partials of 24
 * bytes (3 MiB), which every GPU that loads the library holds until the
 * process exits.  A request needs n_entries x chunks partials when its paths
 * are split into more than one chunk per entry (chunks ~ 77824 / n_entries,
 * at least 1024 paths each); a request beyond 131072 is rejected with
 * MCX_E_UNSUPPORTED before anything is enqueued.
 *
 * The first call on each device looks up the array's device address (with
 * that device current) and caches it; make that first call before any stream
 * capture.  All calls share the array and it keeps the previous call's
 * contents (each call writes every slot it later reads, so nothing needs
 * clearing); calls that overlap on the GPU race on it, so serialise them
 * (one stream, or events between streams).
 * Errors: those of mcx_estimate, plus MCX_E_UNSUPPORTED for oversized requests.
 */
mcx_status mcx_estimate_noalloc(mcx_plan *plan, const double *v, double t, int functional, int32_t nsteps,
                                uint64_t paths_per_entry, const int32_t *entries, int64_t n_entries,
                                uint64_t seed, uint64_t path_offset, int precision, double *mean, double *sem,
                                void *stream);

/*
 * Multilevel Monte Carlo level difference (Giles 2008) for the split
 * functionals (Theorem 1 with Eqs. deff / eq_general1): per requested entry
 * the mean and standard error of Y = v_{X_t} (W_N - W_{N/2}) over
 * paths_per_entry paths, where W_N and W_{N/2} are the STRANG or LIE
 * functionals with N and N/2 steps evaluated on the same path.  The paths are
 * those of mcx_estimate with the same seed and path_offset (the draw schedule
 * does not depend on N), so estimate(N_0) + the differences at N_1 .. N_L on
 * common paths telescope to estimate(N_L); independent levels take disjoint
 * path_offset ranges.
 *   functional       MCX_STRANG or MCX_LIE
 *   nsteps           N, even, >= 2
 *   other arguments  as for mcx_estimate
 * Chunk partials (n_entries x chunks x 24 bytes) come from the library's
 * memory pool, stream-ordered.  An invalid entry yields NaN and MCX_E_INVALID
 * at mcx_sync.
 * Errors: MCX_E_INVALID (also for EXACT or an odd N), MCX_E_CUDA, MCX_E_OOM.
 */
mcx_status mcx_estimate_level_difference(mcx_plan *plan, const double *v, double t, int functional, int32_t nsteps,
                                         uint64_t paths_per_entry, const int32_t *entries, int64_t n_entries,
                                         uint64_t seed, uint64_t path_offset, int precision, double *mean,
                                         double *sem, void *stream);

/*
 * Random-gather ceiling (a measurement for the walkers' roofline: every jump of
 * Sec. 3's path sampler is two gathers, the drawn column and the new state's
 * record, each a random 32-byte sector).  Returns in *sectors_per_second the
 * rate at which this GPU serves `loads` loads of random sectors from a device
 * buffer of `buffer_bytes` (allocated from the library's pool, filled and
 * freed inside the call; 1 MiB <= buffer_bytes <= 128 GiB and fewer than 2^32
 * sectors).  dependent = 1: each thread's next sector depends on the word it
 * loaded (chains of dependent loads, as a walker's jumps are); dependent = 0:
 * independent loads.  One warm-up launch, then one launch timed with CUDA
 * events on `stream`; synchronises the stream.  A buffer that fits in L2
 * measures L2, one far larger than L2 measures HBM.
 * Errors: MCX_E_INVALID, MCX_E_OOM, MCX_E_CUDA.
 */
mcx_status mcx_gather_rate(uint64_t buffer_bytes, int dependent, uint64_t loads, double *sectors_per_second,
                           void *stream);

/* Largest log2 of the points per replicate of mcx_estimate_rqmc. */
#define MCX_QMC_MAX_LOG2 24
/* Sobol' dimensions of mcx_estimate_rqmc: holding time and slot of the first 8 events. */
#define MCX_QMC_DIMS 16

/*
 * Randomised quasi-Monte Carlo backward estimate (the walker of mcx_estimate
 * with quasi-random draws; variance reduction, Sec. 5).  For each requested
 * entry, `replicates` independent randomisations of the first
 * 2^log2_points points of a Sobol' sequence drive the paths: event k < 8 of
 * point q takes its holding-time uniform from Sobol' dimension 2k and its
 * slot uniform from dimension 2k + 1; later events, the FP64 low bits and
 * the alias acceptance keep the path's Philox draws (path index
 * r 2^log2_points + q for replicate r).  Each replicate scrambles the direction
 * numbers with a random lower-triangular binary matrix (Matousek's linear
 * scramble, one per replicate and dimension) and XORs a random digital shift
 * (one per entry, replicate and dimension); the Sobol' parameters are the
 * first entries of Joe and Kuo's table.  Every path is an exact sample of the
 * chain, so each replicate mean mu_r of W v_{X_t} is unbiased.
 *   v, t, functional, nsteps, entries, n_entries, seed, precision
 *                    as for mcx_estimate
 *   log2_points      points per replicate 2^log2_points, 0 <= log2_points <=
 *                    MCX_QMC_MAX_LOG2 (0: one point, a plain Monte Carlo draw)
 *   replicates       1 <= R <= 2^16 (R >= 2 for a standard error); paths per
 *                    entry are R 2^log2_points, at most 2^40
 *   replicate_offset the replicates drawn are replicate_offset ..
 *                    replicate_offset + R - 1 (their scrambles, shifts and
 *                    Philox path indices), so disjoint ranges are independent
 *                    and merge into one estimate (sharding; the sum with R must
 *                    stay below 2^32)
 *   mean             float64 [n_entries] output: the mean of the mu_r
 *   sem              float64 [n_entries] output, or NULL: sqrt(s^2 / R) with
 *                    s^2 the unbiased sample variance of the mu_r (0 if R = 1)
 * Device scratch of R * 16 * ceil(log2_points / 5) * 32 uint32 (digit tables
 * of the scrambled points) and, when n_entries < 77824 (then a warp holds
 * fewer than all replicates of its entry), n_entries * R * slices double
 * pairs comes from the library's memory pool, stream-ordered.  The plan's copy
 * of v is overwritten as in mcx_estimate.  An invalid entry yields NaN and MCX_E_INVALID at
 * mcx_sync; a non-finite result sets the overflow flag.
 * Errors: MCX_E_INVALID, MCX_E_CUDA, MCX_E_OOM.
 */
mcx_status mcx_estimate_rqmc(mcx_plan *plan, const double *v, double t, int functional, int32_t nsteps,
                             uint32_t log2_points, uint32_t replicates, uint32_t replicate_offset,
                             const int32_t *entries, int64_t n_entries, uint64_t seed, int precision, double *mean,
                             double *sem, void *stream);

/*
 * Per-path record of `count` backward paths of one entry (for parity checks
 * against an independent implementation of the same draw schedule):
 *   end     int32  [count]  X_t
 *   njumps  uint32 [count]  number of jumps
 *   hash    uint64 [count]  FNV-1a 64 over the visited indices, start included
 *   logw    float64[count]  log of the multiplicative functional (FP32 paths
 *                           are widened exactly)
 * Paths first_path .. first_path+count-1 of `entry` with the same arguments as
 * mcx_estimate.  Errors: MCX_E_INVALID, MCX_E_CUDA.
 */
mcx_status mcx_trace_paths(mcx_plan *plan, double t, int functional, int32_t nsteps, int32_t entry,
                           uint64_t seed, uint64_t first_path, uint32_t count, int precision,
                           int32_t *end, uint32_t *njumps, uint64_t *hash, double *logw, void *stream);

/*
 * Largest eigenvalue of a symmetric A >= 0 by the power method (Sec. 6 picks
 * beta = 1/lambda_max): x <- A x / ||A x||_2 from x = 1/sqrt(n), Rayleigh
 * quotient x^T A x, stopped when two successive quotients agree to `tol`
 * relative or after max_iters.  Works on the caller's CSR (device pointers,
 * same layout as mcx_plan_create, which must be valid: this call does not
 * re-validate it) with `work` a caller-owned device buffer of at least
 * 3n+4096 float64.  Rows longer than 32 entries (hubs) are handled one warp
 * per row.  *lambda_out and *iters_out (either may be NULL)
 * are host outputs; the call synchronises the stream.
 * Errors: MCX_E_INVALID, MCX_E_CUDA.
 */
mcx_status mcx_power_iteration(int64_t n, const int64_t *row_ptr, const int32_t *col, const double *val,
                               int32_t max_iters, double tol, double *work, double *lambda_out,
                               int32_t *iters_out, void *stream);

/*
 * Multilevel combination (Giles' telescoping sum over the step count of the
 * STRANG/LIE functionals, the multilevel reading of the split error of Sec. 5):
 * per entry, mean = the sum of the level means in level order (level 0 the
 * plain estimate with N_0 steps, level l the level difference N_l vs N_l/2),
 * sem = the square root of the sum of the squared level standard errors (the
 * levels use disjoint path ranges, so they are independent).
 *   levels       1 .. 64
 *   means, sems  host arrays of `levels` device pointers, each float64
 *                [n_entries]; sems may be NULL when sem is NULL
 *   mean, sem    float64 [n_entries] device outputs (sem may be NULL)
 * Asynchronous on `stream`.  Errors: MCX_E_INVALID, MCX_E_CUDA.
 */
mcx_status mcx_combine_levels(int32_t levels, int64_t n_entries, const double *const *means,
                              const double *const *sems, double *mean, double *sem, void *stream);

/*
 * Copy the plan's preparation results (Sec. 2 decomposition, Sec. 4 jump
 * tables) into caller-owned device arrays, for parity checks against an
 * independent preparation.  Per row [n]: deg (int32), row_start (int64),
 * weighted (uint8, 1 for alias-table rows), inv_rate32 = (float)(1/lambda),
 * delta32 = (float)delta, inv_rate64, delta64 (float64).  Per kept entry
 * [nnz_off] (mcx_plan_info): edge_col (int32, CSR order), alias_col (int32),
 * thresh (uint32); for uniform rows alias_col = edge_col and thresh =
 * 0xFFFFFFFF.  Any output may be NULL.  Errors: MCX_E_INVALID, MCX_E_CUDA.
 */
mcx_status mcx_plan_export(const mcx_plan *plan, int32_t *deg, int64_t *row_start, uint8_t *weighted,
                           float *inv_rate32, float *delta32, double *inv_rate64, double *delta64,
                           int32_t *edge_col, int32_t *alias_col, uint32_t *thresh, void *stream);

/* ------------------------------------------------------------------------ */
/* Batching: many forward problems in one persistent launch.                */
/* ------------------------------------------------------------------------ */
typedef struct mcx_batch mcx_batch;

/* One forward problem (host memory): the plan matrix B = A^T in CSR form (as
 * for mcx_plan_create), v >= 0 [n], n_times horizons t > 0, and `paths`
 * forward paths for each horizon. */
typedef struct {
    int64_t n;
    int64_t nnz;
    const int64_t *row_ptr;
    const int32_t *col;
    const double *val;
    const double *v;
    int32_t n_times;
    const double *times;
    uint64_t paths;
} mcx_problem;

typedef struct {
    int32_t problems;        /* problems in the batch */
    int32_t pairs;           /* (problem, time) pairs */
    int64_t states;          /* states of the block-diagonal plan, blocks padded to multiples of 1024 */
    uint64_t total_paths;    /* paths per run */
    uint32_t work_items;     /* work items per run */
    uint32_t chunk;          /* paths per work item (autotuned) */
    int32_t blocks_per_sm;   /* resident blocks of 256 threads per SM (autotuned) */
    int32_t grid;            /* persistent grid size */
    int32_t count_deposits;  /* 1: every potential is zero, deposits are exact counts */
    int32_t lane_refill;     /* 1: lanes take the next path of the item as theirs end (autotuned) */
    double tuned_ms;         /* the autotuner's best sampled run (0 if read from the cache) */
} mcx_batch_info;

/*
 * Build a batch of forward problems (Theorem 2, Algorithm 2) for one
 * persistent launch.  The matrices are placed on the diagonal of one plan
 * (blocks padded to multiples of 1024 states), per-problem two-level start
 * tables are built over each v, and the (problem, time) pairs are cut into
 * work items ordered by estimated cost (largest first: cost ~ paths x
 * (1 + t x mean jump rate)).  The schedule (paths per work item, resident
 * blocks per SM, lane refill on or off) is read from `tune_cache` (a file of
 * JSON lines keyed by GPU
 * name and problem-set sizes; NULL: no cache) or autotuned by timing sampled
 * runs, then appended to the cache.  The reset + start tables + walk +
 * finish sequence is captured into a CUDA graph.  Pair k of the batch uses path indices
 * k * 2^40 + p (pairs numbered problem by problem, time by time), so its
 * paths are those of mcx_estimate_forward on that problem alone with
 * path_offset = k * 2^40.  EXACT functional, FP32 paths.  Synchronises
 * `stream`.
 * Errors: MCX_E_INVALID (bad description or CSR), MCX_E_NEG_OFFDIAG,
 * MCX_E_NONFINITE, MCX_E_NEG_V (some v invalid), MCX_E_OOM, MCX_E_CUDA.
 */
mcx_status mcx_batch_create(int32_t count, const mcx_problem *problems, const char *tune_cache, void *stream,
                            mcx_batch **out);

/* One run of the whole batch (one graph launch) with the given seed; results
 * replace the previous run's.  Asynchronous on `stream`. */
mcx_status mcx_batch_run(mcx_batch *batch, uint64_t seed, void *stream);

/* Replace the start vector of problem `problem` (device float64 [n], >= 0 with a
 * positive sum) for the next runs: every run's graph rebuilds the start tables
 * (Lemma 2) from the batch's current values, so no re-creation is needed.  An
 * invalid v is found on the device: that run's results are NaN and
 * mcx_batch_sync returns MCX_E_NEG_V.  Asynchronous on `stream`.
 * Errors: MCX_E_INVALID, MCX_E_CUDA. */
mcx_status mcx_batch_set_v(mcx_batch *batch, int32_t problem, const double *v, void *stream);

/* Copy the last run's estimate of problem `problem` at horizon `time_index`
 * into caller-owned device arrays x [n] and sem [n] (sem may be NULL).
 * Errors: MCX_E_INVALID, MCX_E_CUDA. */
mcx_status mcx_batch_result(const mcx_batch *batch, int32_t problem, int32_t time_index, double *x, double *sem,
                            void *stream);

/* Fill *info (host) with the batch's layout and schedule. */
mcx_status mcx_batch_get_info(const mcx_batch *batch, mcx_batch_info *info);

/* mcx_sync for the batch's plan (latched status, path and jump counters). */
mcx_status mcx_batch_sync(mcx_batch *batch, void *stream, mcx_stats *stats);

/* Free the batch (synchronises the device first).  NULL is accepted. */
void mcx_batch_destroy(mcx_batch *batch);

/* ------------------------------------------------------------------------ */
/* Learned control variate (variance reduction, Sec. 5).                    */
/*                                                                          */
/* For any h with h(0) = v, x_i = h(t, i) + E_i[int_0^t W_s R(t - s, X_s) ds] */
/* with R = A h - dh/dtau (Duhamel's formula with the Feynman-Kac form of    */
/* exp(sA), Theorem 1): unbiased whatever h is.  The library uses            */
/* h(tau) = v + tau Av + tau^2 A^2 v/2 + tau^3 c3 with c3 chosen so that       */
/* h(t, i) = xhat_i, a prediction of x_i by a small network; then            */
/* R(tau) = a tau^2 + b tau^3, a = A^3 v/2 - 3 c3, b = A c3, and the walker    */
/* integrates e^{logW} R exactly over every holding interval.  A good        */
/* prediction leaves only a small residual to estimate.                     */
/* ------------------------------------------------------------------------ */
typedef struct mcx_mlp mcx_mlp;

/*
 * Taylor terms and node features of (A, v, t); all pointers are device memory.
 *   taylor   float64 [4n] out: v, Av, A^2 v, A^3 v (A with its diagonal)
 *   features float32 [5n] out, node-major: log1p(lambda_i), log1p(mean of the
 *            neighbours' lambda), log1p(their standard deviation),
 *            t(Av)_i/T2_i, t^2(A^2v)_i/(2 T2_i), T2 = v + tAv + t^2A^2v/2
 *   work     float64 [3n + 64] scratch, 16-byte aligned
 * Two passes over the rows form Av with the rates lambda, then A^2 v with the
 * features; a third forms A^3 v.  Rows longer than 32 entries (hubs) are
 * handled one warp per row, rows longer than 1024 one block per row.
 * Errors: MCX_E_INVALID (also a misaligned work), MCX_E_CUDA.
 */
mcx_status mcx_cv_prepare(int64_t n, const int64_t *row_ptr, const int32_t *col, const double *val,
                          const double *v, double t, double *work, double *taylor, float *features, void *stream);

/* Training targets y_i = log(max(x_i / T2_i, 1e-6)) from estimates x (float64 [n])
 * and the Taylor terms; y float32 [n] out (device). */
mcx_status mcx_cv_targets(int64_t n, const double *x, const double *taylor, double t, float *y, void *stream);

/* A 5-64-64-1 ReLU network predicting y = log(x / T2) from the features
 * (standardised with the training set's mean and deviation).  FP32 master
 * weights on the device; every use rounds the weights to BF16 (round to
 * nearest even) and accumulates in FP32.  Initialised from `seed`. */
mcx_status mcx_mlp_create(uint64_t seed, mcx_mlp **out);

/* Host copies of the parameters (4609 floats: W1 [5][64] in-major, b1 [64],
 * W2 [64][64], b2 [64], W3 [64], b3) and the feature mean / deviation [5];
 * any pointer may be NULL. */
mcx_status mcx_mlp_set(mcx_mlp *model, const float *params, const float *mu, const float *sd);
mcx_status mcx_mlp_get(const mcx_mlp *model, float *params, float *mu, float *sd);

/* y [n] = network(features [5n]) (device), on the tensor cores: tiles of 128
 * nodes; the first hidden layer (FP32, BF16 weights) is rounded to BF16 (round
 * to nearest even) and multiplied by W2 (BF16) with FP32 accumulation in
 * tensor memory (tcgen05 MMAs); bias, ReLU and the output layer in FP32.
 * Asynchronous; a device-side failure of an MMA completion wait is latched and
 * returned by mcx_mlp_sync. */
mcx_status mcx_mlp_predict(const mcx_mlp *model, int64_t n, const float *features, float *y, void *stream);

/* Synchronise `stream`; return and clear the model's latched device status
 * (inference and training): MCX_OK, or MCX_E_TIMEOUT if an MMA completion wait
 * gave up (that call's outputs, or the training step's gradient, are
 * unspecified).  Errors: MCX_E_INVALID, MCX_E_CUDA. */
mcx_status mcx_mlp_sync(mcx_mlp *model, void *stream);

/* Gradient of the mean squared error (1/n) sum (net(f_i) - y_i)^2 with respect
 * to the parameters as used (BF16-rounded weights): grad float32 [4609]
 * (device) and the loss (host, may be NULL; the call then synchronises).  On
 * the tensor cores, tiles of 128 samples: the forward pass as in
 * mcx_mlp_predict (h1 rounded to BF16); the hidden layer's backward signal
 * dh2 = dy W3 [z2 > 0] rounded to BF16 (round to nearest even); dh1 = dh2 W2^T
 * and dW2 = h1^T dh2, db2 = sum dh2 as BF16 MMAs with FP32 accumulation in
 * tensor memory; dW1, db1, dW3, db3 and the loss in FP32 on CUDA cores.
 * Deterministic: tile partial sums are added in a fixed order.  A device-side
 * failure of an MMA completion wait is latched for mcx_mlp_sync. */
mcx_status mcx_mlp_gradient(mcx_mlp *model, int64_t n, const float *features, const float *targets,
                            float *grad, float *loss, void *stream);

/* Adam (beta1 0.9, beta2 0.999, eps 1e-8, learning rate lr) on minibatches of
 * `batch` rows (gradients as mcx_mlp_gradient computes them), `epochs` passes
 * over a permutation drawn from `seed`; first sets the feature standardisation
 * from these features.  epoch_loss (host,
 * [epochs], may be NULL) receives the mean minibatch loss of each epoch.
 * Synchronises `stream`. */
mcx_status mcx_mlp_fit(mcx_mlp *model, int64_t n, const float *features, const float *targets, int32_t epochs,
                       int32_t batch, float lr, uint64_t seed, float *epoch_loss, void *stream);

void mcx_mlp_destroy(mcx_mlp *model);

/*
 * Control-variate coefficients from the Taylor terms and the network output
 * y (float32 [n], device; NULL means y = 0, i.e. xhat = T2, the Taylor-only
 * control variate): coef float64 [3n] out = [(a_i, b_i) pairs (2n) | h (n)]
 * with h_i = xhat_i = T2_i e^{y_i}, c3 = (xhat - T2)/t^3, a = A^3 v/2 - 3 c3,
 * b = A c3; coef must be 16-byte aligned (the pairs are read as 16-byte
 * vectors).  work: float64 [3n + 64] scratch.  Errors: MCX_E_INVALID, MCX_E_CUDA.
 */
mcx_status mcx_cv_coefficients(int64_t n, const int64_t *row_ptr, const int32_t *col, const double *val,
                               const double *taylor, const float *y, double t, double *work, double *coef,
                               void *stream);

/*
 * Control-variate backward estimate of x_i = (exp(tA) v)_i for the requested
 * entries: mean = h_i + the sample mean of the residual integrals over
 * `paths` paths (the FP32 paths of mcx_estimate with the same seed, EXACT
 * functional), sem = the residuals' standard error.  precision: MCX_FP32
 * (residual integrals in FP32 with per-path scaling) or MCX_FP64 (in FP64).
 * coef from mcx_cv_coefficients for the same (A, v, t); entries, outputs and
 * errors as in mcx_estimate.
 */
mcx_status mcx_estimate_cv(mcx_plan *plan, const double *coef, double t, uint64_t paths, const int32_t *entries,
                           int64_t n_entries, uint64_t seed, uint64_t path_offset, int precision, double *mean,
                           double *sem, void *stream);

/* ------------------------------------------------------------------------ */
/* Batched backward estimates with the control variate (Theorem 1,          */
/* Algorithm 1; variance reduction of Sec. 5): many (A, v, t), several      */
/* right-hand sides per A, the whole full-vector computation of every       */
/* (problem, right-hand side) pair in one CUDA-graph launch: per pair the   */
/* Taylor terms, features, network prediction and coefficients (the        */
/* pre-pass), then one persistent walk over a work list of (pair, entries,  */
/* path chunk) items, then the per-entry finish.                            */
/* ------------------------------------------------------------------------ */
typedef struct mcx_cvbatch mcx_cvbatch;

typedef enum {
    MCX_CV_NONE = 0,     /* plain backward estimate: mean of W v_{X_t} (the reference for the others) */
    MCX_CV_TAYLOR = 1,   /* control variate with h(t) = the second-order Taylor term T2 */
    MCX_CV_LEARNED = 2   /* control variate with h(t) = the network's prediction */
} mcx_cv_control;

/* One matrix of a control-variate batch (host memory, read during create). */
typedef struct {
    int64_t n, nnz;           /* A is n x n with nnz stored entries (CSR as for mcx_plan_create) */
    const int64_t *row_ptr;   /* int64 [n+1] */
    const int32_t *col;       /* int32 [nnz] */
    const double *val;        /* float64 [nnz] */
    int32_t n_rhs;            /* right-hand sides of this A (>= 1) */
    const double *v;          /* float64 [n_rhs * n]: right-hand side r at v + r n */
    const double *t;          /* float64 [n_rhs]: horizon of each right-hand side, > 0 and finite */
    uint64_t paths;           /* paths per entry, 1 .. 2^40 */
} mcx_cv_problem;

typedef struct {
    int32_t problems;        /* problems in the batch */
    int32_t pairs;           /* (problem, right-hand side) pairs */
    int64_t states;          /* states of the block-diagonal plan, blocks padded to multiples of 1024 */
    uint64_t total_paths;    /* paths per run */
    uint32_t work_items;     /* work items per run */
    uint32_t chunk;          /* paths per work item of the warp-per-entry layout (autotuned) */
    int32_t blocks_per_sm;   /* resident blocks of 256 threads per SM (autotuned) */
    int32_t grid;            /* persistent grid size */
    int32_t staged;          /* 1: warps stage their entry's row in shared memory (autotuned) */
    int32_t control;         /* mcx_cv_control */
    double tuned_ms;         /* the autotuner's best sampled walk (0 if read from the cache) */
} mcx_cvbatch_info;

/*
 * Build a batch of backward full-vector estimates.  The matrices go on the
 * diagonal of one plan (blocks padded to multiples of 1024 states); each pair
 * (problem b, right-hand side r), numbered problem by problem, keeps its own
 * v, t, Taylor terms, features, prediction and coefficients.  Every entry of
 * every pair is estimated with the problem's `paths`: pairs with at most 64
 * paths per entry run one lane per entry (items of 32 entries), the others one
 * warp per (entry, chunk of paths) with lane refill; items are ordered by
 * estimated cost, largest first (cost ~ paths x (1 + t x mean jump rate)), and
 * taken from an atomic counter by a persistent grid.  The schedule (chunk
 * length, resident blocks per SM, staging of each warp's entry row in shared
 * memory) is read from `tune_cache` (JSON lines keyed by GPU name and
 * batch sizes; NULL: no cache) or autotuned by timing the walk on a sample of
 * the items, then appended to the cache.
 *   control    mcx_cv_control; MCX_CV_LEARNED needs `net`, whose weights are
 *              read at every run (retraining it between runs is allowed)
 *   precision  MCX_CV_NONE: MCX_FP32 (FP32 paths, compensated FP32 sums) or
 *              MCX_FP64 (the FP64 path version); control variates: FP32
 *              paths with the residual integrals in FP32 or FP64 (as in
 *              mcx_estimate_cv)
 * Pair k of the batch simulates paths k * 2^40 + p (p = 0 .. paths-1) of each
 * entry, i.e. exactly the paths of mcx_estimate (MCX_CV_NONE) or
 * mcx_estimate_cv on that problem alone with path_offset = k * 2^40 and the
 * run's seed (EXACT functional).  Synchronises `stream`.
 * Limits: the problems' states (each padded to a multiple of 1024) and the
 * slots (sum over pairs of n) must each stay below 2^31 - 1.
 * Errors: MCX_E_INVALID (bad description or CSR, missing net, a limit
 * exceeded), MCX_E_NEG_OFFDIAG, MCX_E_NONFINITE, MCX_E_OOM, MCX_E_CUDA.
 */
mcx_status mcx_cvbatch_create(int32_t count, const mcx_cv_problem *problems, int control, const mcx_mlp *net,
                              int precision, const char *tune_cache, void *stream, mcx_cvbatch **out);

/* Change the paths per entry of every problem (host uint64 [problems]); the
 * work list is rebuilt and the graph re-captured with the current schedule.
 * Synchronises `stream`.  Errors: MCX_E_INVALID, MCX_E_OOM, MCX_E_CUDA. */
mcx_status mcx_cvbatch_set_paths(mcx_cvbatch *batch, const uint64_t *paths, void *stream);

/* One run of the whole batch (one graph launch: pre-pass, walk, finish) with
 * the given seed; results replace the previous run's.  Asynchronous on `stream`. */
mcx_status mcx_cvbatch_run(mcx_cvbatch *batch, uint64_t seed, void *stream);

/* Copy the last run's estimate of (problem, rhs) into caller-owned device
 * arrays x [n] and sem [n] (sem may be NULL).  Errors: MCX_E_INVALID, MCX_E_CUDA. */
mcx_status mcx_cvbatch_result(const mcx_cvbatch *batch, int32_t problem, int32_t rhs, double *x, double *sem,
                              void *stream);

/* Copy the last run's control-variate coefficients of (problem, rhs), laid
 * out as mcx_cv_coefficients writes them, float64 [3n] device
 * = [(a, b) pairs | h].  Errors: MCX_E_INVALID (also for MCX_CV_NONE), MCX_E_CUDA. */
mcx_status mcx_cvbatch_coefficients(const mcx_cvbatch *batch, int32_t problem, int32_t rhs, double *coef,
                                    void *stream);

/* Fill *info (host) with the batch's layout and schedule. */
mcx_status mcx_cvbatch_get_info(const mcx_cvbatch *batch, mcx_cvbatch_info *info);

/* mcx_sync for the batch's plan; with MCX_CV_LEARNED also the network's
 * latched inference status (MCX_E_TIMEOUT if a tensor-core wait gave up). */
mcx_status mcx_cvbatch_sync(mcx_cvbatch *batch, void *stream, mcx_stats *stats);

/* Free the batch (synchronises the device first).  NULL is accepted. */
void mcx_cvbatch_destroy(mcx_cvbatch *batch);

/* Synchronise `stream`, return and clear the plan's latched device status and
 * counters.  stats (host pointer) may be NULL.  Errors: MCX_E_INVALID (an
 * estimate was given an entry outside [0, n); its outputs are NaN),
 * MCX_E_NEG_V (a forward call got v with a negative or non-finite entry or a
 * zero sum; its outputs are NaN),
 * MCX_E_OVERFLOW (a result overflowed FP64, or a path reached the cap of 2^30
 * events), MCX_E_CUDA. */
mcx_status mcx_sync(mcx_plan *plan, void *stream, mcx_stats *stats);

/* Free the plan's device memory (synchronises the device first).  NULL is accepted. */
void mcx_plan_destroy(mcx_plan *plan);

/* Static string for a status code. */
const char *mcx_status_string(int status);

/*
 * Test hooks for the failure paths (the paper has no counterpart; not for
 * production use).  mcx_debug_fail_alloc(k): the k-th device allocation the
 * library makes from now on (pool or cudaMalloc) fails as if the device were
 * out of memory, so that the call making it returns MCX_E_OOM; k <= 0
 * disarms.  Returns the number of device allocations the library has
 * attempted since the process started.  mcx_debug_pool_usage: bytes of the
 * library's memory pool on the current device in use and reserved (host
 * outputs, either may be NULL), to check that failed calls leak nothing.
 */
int64_t mcx_debug_fail_alloc(int64_t k);
mcx_status mcx_debug_pool_usage(uint64_t *used, uint64_t *reserved);

/* Test hook: the polls the network's tensor-core kernels (inference and
 * gradient) spend waiting for the MMAs of a tile before they give up (default 2^22; 0xFFFFFFFF restores the
 * default).  With 0 every wait gives up at once: the kernel latches the error
 * (mcx_mlp_sync returns MCX_E_TIMEOUT), waits with the default limit for the
 * MMAs it has in flight, frees its tensor memory and returns; nothing traps.
 * Errors: MCX_E_INVALID. */
mcx_status mcx_debug_mlp_wait_polls(mcx_mlp *model, uint32_t polls);

/* Library version as 10000*major + 100*minor + patch. */
int mcx_version(void);

#ifdef __cplusplus
}
#endif

#endif /* MCX_H */
