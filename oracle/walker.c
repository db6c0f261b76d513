/*
 * CPU oracle walker for the Monte Carlo exp(tA)v estimator.
 *
 * TEST INFRASTRUCTURE ONLY: called by the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark.  It shares no code with the CUDA library;
 * it is a plain, sequential statement of the paper's method:
 *
 *   - A = D - L (Sec. 2): the potential delta_i is the full row sum of A, the
 *     jump rate lambda_i = sum_{j != i} a_ij is L_ii, and -L is the generator
 *     of the continuous-time Markov chain (Lemma 1).
 *   - Path sampler (Sec. 3, Eq. paths): exponential holding times with rate
 *     lambda_j, jumps with probability k_ij = a_ij / lambda_j, stop at the
 *     horizon t.
 *   - Multiplicative functional (Theorem 1; Algorithm 1): the weight
 *     W = exp(logW) with logW = integral of delta along the path (EXACT), or
 *     its Lie / Strang quadratures on the grid k*dt, dt = t/N (Eqs. deff and
 *     eq_general1).  The estimate of entry i is the sample mean of W v_{X_t}.
 *   - Forward form (Lemma 2, Theorem 2; Algorithm 2): start j ~ v/V, deposit
 *     V W at the end state.
 *
 * Build: gcc -O2 -ffp-contract=off -fno-fast-math -fopenmp -shared -fPIC.
 * Every floating-point operation below is a single IEEE operation or an
 * explicit fma, so the result does not depend on the compiler's contraction
 * choices.
 *
 * Draw schedule (fixed so that another implementation can reproduce every
 * path exactly): one Philox4x32-10 call per walker event, key = seed,
 * counter = {event k, entry i, path lo32, path hi32}.  Word 0 (and word 1 in
 * FP64) gives the holding-time uniform, word 2 the slot in the row, word 3 the
 * alias acceptance.  The randomised-QMC estimator replaces words 0 and 2 of the
 * first events by scrambled Sobol' coordinates (see below); the multilevel
 * level difference runs each path twice, at N and N/2 steps, on the same draws.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define O_EXACT 0
#define O_STRANG 1
#define O_LIE 2

/* ------------------------------------------------------------------------ */
/* Philox4x32-10: Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as   */
/* easy as 1, 2, 3", SC'11.  Ten rounds of two 32x32->64 multiplies; the key */
/* is bumped by the Weyl constants between rounds.                           */
/* ------------------------------------------------------------------------ */
void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)x0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
        uint32_t y0 = (uint32_t)(p1 >> 32) ^ x1 ^ k0;
        uint32_t y1 = (uint32_t)p1;
        uint32_t y2 = (uint32_t)(p0 >> 32) ^ x3 ^ k1;
        uint32_t y3 = (uint32_t)p0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

static void draw(uint64_t seed, uint32_t event, uint32_t stream, uint64_t path, uint32_t w[4])
{
    uint32_t ctr[4] = {event, stream, (uint32_t)path, (uint32_t)(path >> 32)};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    oracle_philox4x32_10(ctr, key, w);
}

/* Uniforms in (0, 1]: never zero, so the logarithm below is always finite. */
static float unif_f32(uint32_t w0) { return (float)(16777216u - (w0 >> 8)) * 0x1p-24f; }
static double unif_f64(uint32_t w0, uint32_t w1)
{
    uint64_t m = ((uint64_t)w0 << 21) | (uint64_t)(w1 >> 11);
    return (double)(9007199254740992ull - m) * 0x1p-53;
}

/* ------------------------------------------------------------------------ */
/* FP32 natural logarithm, table-driven (P. T. P. Tang, "Table-driven         */
/* implementation of the logarithm function in IEEE floating-point            */
/* arithmetic", ACM TOMS 16(4), 1990), with no division.  Write x = 2^E M,    */
/* M in [1, 2).  The breakpoints are c_j = 1 + j/64, j = 0..64; j is the one  */
/* nearest M (the top six mantissa bits, rounded).  With inv_j = 1/c_j in     */
/* FP32, r = M inv_j - 1 (one fma; |r| <= 2^-7) and                           */
/*     ln x = E ln2 + ln(1/inv_j) + ln(1 + r),                                */
/* ln(1 + r) by its Taylor polynomial r - r^2/2 + r^3/3 - r^4/4.  Rows with   */
/* c_j > sqrt2 (j >= 27) move one factor 2 into the exponent (E + 1 and       */
/* ln(1/(2 inv_j))), so the table term stays below ln sqrt2 in size and      */
/* x near 1 (E = -1, M near 2) loses nothing to cancellation.                 */
/* ------------------------------------------------------------------------ */
#define LN_ROWS 65
#define LN_SPLIT 27
static float ln_inv[LN_ROWS], ln_row[LN_ROWS];

/* Filled when the library is loaded, before any walker thread runs. */
__attribute__((constructor)) static void ln_table_init(void)
{
    for (int j = 0; j < LN_ROWS; ++j) {
        float inv = (float)(1.0 / (1.0 + (double)j / 64.0));
        double a = j >= LN_SPLIT ? 2.0 * (double)inv : (double)inv;
        ln_inv[j] = inv;
        ln_row[j] = (float)(0.0 - log(a));
    }
}

/* The table as the logarithm uses it (for the tests): inv[j], L[j]. */
void oracle_ln_table(float *inv, float *L)
{
    for (int j = 0; j < LN_ROWS; ++j) {
        inv[j] = ln_inv[j];
        L[j] = ln_row[j];
    }
}

float oracle_logf(float x)
{
    uint32_t b;
    memcpy(&b, &x, 4);
    uint32_t mb = b & 0x007fffffu;
    int j = (int)((mb + 0x10000u) >> 17);
    int e = (int)(b >> 23) - 127 + (j >= LN_SPLIT ? 1 : 0);
    uint32_t mbits = mb | 0x3f800000u;
    float m;
    memcpy(&m, &mbits, 4);
    float r = fmaf(m, ln_inv[j], -1.0f);
    float q = fmaf(r, -0.25f, 1.0f / 3.0f);
    q = fmaf(q, r, -0.5f);
    float p = fmaf(r * r, q, r);
    return fmaf((float)e, 0.693147181f, ln_row[j]) + p;
}

/* Batch form for the tests: y[k] = oracle_logf(x[k]). */
void oracle_logf_many(const float *x, float *y, int64_t n)
{
    for (int64_t k = 0; k < n; ++k) y[k] = oracle_logf(x[k]);
}

/* ------------------------------------------------------------------------ */
/* FP64 natural logarithm by range reduction x = 2^e m, m in [1/sqrt2,      */
/* sqrt2], and the series ln m = 2 artanh(s) = 2 (s + s^3/3 + s^5/5 + ...),  */
/* s = (m-1)/(m+1) (Abramowitz & Stegun 4.1.27).  Valid for positive normal  */
/* finite x.                                                                 */
/* ------------------------------------------------------------------------ */
double oracle_log(double x)
{
    uint64_t b;
    memcpy(&b, &x, 8);
    int e = (int)((b >> 52) & 0x7ffu) - 1023;
    uint64_t mb = (b & 0x000fffffffffffffull) | 0x3ff0000000000000ull;
    double m;
    memcpy(&m, &mb, 8);
    if (m > 1.4142135623730951) {
        m = m * 0.5;
        e = e + 1;
    }
    double s = (m - 1.0) / (m + 1.0);
    double z = s * s;
    double q = 1.0 / 25.0;
    q = fma(q, z, 1.0 / 23.0);
    q = fma(q, z, 1.0 / 21.0);
    q = fma(q, z, 1.0 / 19.0);
    q = fma(q, z, 1.0 / 17.0);
    q = fma(q, z, 1.0 / 15.0);
    q = fma(q, z, 1.0 / 13.0);
    q = fma(q, z, 1.0 / 11.0);
    q = fma(q, z, 1.0 / 9.0);
    q = fma(q, z, 1.0 / 7.0);
    q = fma(q, z, 1.0 / 5.0);
    q = fma(q, z, 1.0 / 3.0);
    double s2 = s + s;
    double lnm = fma(s2 * z, q, s2);
    return fma((double)e, 0.6931471805599453, lnm);
}

/* ------------------------------------------------------------------------ */
/* Preparation: the decomposition A = D - L of Sec. 2 and the jump tables.   */
/* ------------------------------------------------------------------------ */
typedef struct {
    int64_t n;
    int64_t nnz_off;
    int32_t *deg;        /* kept off-diagonal entries (a_ij > 0, j != i) */
    int64_t *row_start;  /* exclusive prefix sum of deg */
    uint8_t *weighted;   /* 1 if the kept entries are not all bit-equal */
    float *inv_rate32;   /* (float)(1/lambda_i) */
    float *delta32;      /* (float)delta_i */
    double *inv_rate64;  /* 1/lambda_i */
    double *delta64;     /* delta_i = a_ii + lambda_i */
    int32_t *edge_col;   /* kept columns, CSR order */
    int32_t *alias_col;  /* weighted rows: alias column of each slot */
    uint32_t *thresh;    /* weighted rows: keep the slot's own column iff word3 < thresh */
} oracle_graph;

/* Status codes (mirroring the library's meaning, defined independently). */
#define O_OK 0
#define O_E_INVALID -1
#define O_E_NEG_OFFDIAG -2
#define O_E_NONFINITE -3

/* Canonical Vose alias construction for one row of weights a[0..d-1] with
 * sum lam.  Scaled weights q_k = (a_k d)/lam; indices with q < 1 go to the
 * "small" list and the rest to "large", both in index order; pairs are popped
 * from the back; the large entry keeps (q_l + q_s) - 1.  Leftovers get
 * probability 1 and alias themselves.  The probability is stored as the
 * 32-bit threshold floor(q * 2^32). */
static void vose_row(int d, const double *a, double lam, const int32_t *cols,
                     int32_t *alias_out, uint32_t *thresh_out, double *q, int *small, int *large)
{
    int ns = 0, nl = 0;
    for (int k = 0; k < d; ++k) {
        q[k] = (a[k] * (double)d) / lam;
        if (q[k] < 1.0) small[ns++] = k;
        else large[nl++] = k;
    }
    for (int k = 0; k < d; ++k) {
        alias_out[k] = cols[k];
        thresh_out[k] = 0xFFFFFFFFu;
    }
    while (ns > 0 && nl > 0) {
        int s = small[--ns];
        int l = large[--nl];
        thresh_out[s] = (uint32_t)(q[s] * 4294967296.0);
        alias_out[s] = cols[l];
        q[l] = (q[l] + q[s]) - 1.0;
        if (q[l] < 1.0) small[ns++] = l;
        else large[nl++] = l;
    }
}

int oracle_prep(int64_t n, const int64_t *row_ptr, const int32_t *col, const double *val,
                oracle_graph *g)
{
    /* validation: CSR structure, sorted unique columns, finite values, a_ij >= 0 off the diagonal */
    if (n < 0 || row_ptr[0] != 0) return O_E_INVALID;
    for (int64_t i = 0; i < n; ++i) {
        if (row_ptr[i + 1] < row_ptr[i]) return O_E_INVALID;
        for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) {
            if (col[p] < 0 || col[p] >= n) return O_E_INVALID;
            if (p > row_ptr[i] && col[p] <= col[p - 1]) return O_E_INVALID;
            if (!isfinite(val[p])) return O_E_NONFINITE;
            if (col[p] != i && val[p] < 0.0) return O_E_NEG_OFFDIAG;
        }
    }
    int64_t off = 0;
    for (int64_t i = 0; i < n; ++i) {
        double lam = 0.0, diag = 0.0;
        int d = 0, uniform = 1;
        double first = 0.0;
        for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) {
            if (col[p] == i) {
                diag = val[p];
            } else if (val[p] > 0.0) {
                if (d == 0) first = val[p];
                else if (memcmp(&first, &val[p], 8) != 0) uniform = 0;
                lam += val[p];
                ++d;
            }
        }
        if (!isfinite(lam) || !isfinite(diag + lam) || !isfinite((float)(diag + lam)) ||
            (d > 0 && (float)(1.0 / lam) == 0.0f))
            return O_E_NONFINITE; /* rates/potentials must be finite with a nonzero FP32 reciprocal rate */
        g->deg[i] = d;
        g->row_start[i] = off;
        g->weighted[i] = (uint8_t)(d > 1 && !uniform);
        g->delta64[i] = diag + lam;
        g->delta32[i] = (float)(diag + lam);
        g->inv_rate64[i] = d > 0 ? 1.0 / lam : 0.0;
        g->inv_rate32[i] = (float)g->inv_rate64[i];
        off += d;
    }
    g->nnz_off = off;
    int maxd = 0;
    for (int64_t i = 0; i < n; ++i)
        if (g->deg[i] > maxd) maxd = g->deg[i];
    double *a = (double *)malloc(sizeof(double) * (size_t)(maxd + 1));
    double *q = (double *)malloc(sizeof(double) * (size_t)(maxd + 1));
    int *sm = (int *)malloc(sizeof(int) * (size_t)(maxd + 1));
    int *lg = (int *)malloc(sizeof(int) * (size_t)(maxd + 1));
    for (int64_t i = 0; i < n; ++i) {
        int64_t o = g->row_start[i];
        int d = 0;
        double lam = 0.0;
        for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) {
            if (col[p] != i && val[p] > 0.0) {
                g->edge_col[o + d] = col[p];
                a[d] = val[p];
                lam += val[p];
                ++d;
            }
        }
        if (g->weighted[i]) {
            vose_row(d, a, lam, g->edge_col + o, g->alias_col + o, g->thresh + o, q, sm, lg);
        } else {
            for (int k = 0; k < d; ++k) {
                g->alias_col[o + k] = g->edge_col[o + k];
                g->thresh[o + k] = 0xFFFFFFFFu;
            }
        }
    }
    free(a); free(q); free(sm); free(lg);
    return O_OK;
}

/* Number of edges kept by oracle_prep (to size its output arrays). */
int64_t oracle_count_offdiag(int64_t n, const int64_t *row_ptr, const int32_t *col, const double *val)
{
    int64_t c = 0;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p)
            if (col[p] != i && val[p] > 0.0) ++c;
    return c;
}

/* ------------------------------------------------------------------------ */
/* Quasi-random draws for the first events of a path (randomised QMC, one of */
/* the variance-reduction directions of Sec. 5).                             */
/*                                                                           */
/* Sobol' points (Sobol' 1967; Bratley & Fox 1988): coordinate d of point q  */
/* is the XOR of the direction numbers V_d[b] over the set bits b of q.      */
/* Dimension 0 takes V_0[b] = 2^(31-b) (van der Corput); dimension d >= 1    */
/* takes a primitive polynomial x^s + a_1 x^(s-1) + ... + a_(s-1) x + 1 over */
/* GF(2) and initial odd m_1..m_s (m_k < 2^k), continued by                  */
/*   m_k = 2 a_1 m_(k-1) ^ 4 a_2 m_(k-2) ^ ... ^ 2^s m_(k-s) ^ m_(k-s),       */
/* and V_d[k-1] = m_k 2^(32-k).  The (s, a, m) below are the first entries   */
/* of Joe & Kuo's table (ACM TOMS 29, 2003; SIAM J. Sci. Comput. 30, 2008).  */
/*                                                                           */
/* Randomisation per replicate r: Matousek's (1998) random linear scramble, a */
/* lower-triangular binary matrix L_(r,d) with unit diagonal (output bit b,   */
/* counted from the most significant, depends on input bits 0..b), applied   */
/* to the direction numbers, followed by a random digital shift e_(i,r,d)    */
/* (XOR) per entry i.  Both keep the net structure; every point is uniform,  */
/* so each replicate mean is unbiased and the spread of R independent         */
/* replicate means gives the standard error.                                 */
/*                                                                           */
/* Draw schedule: event k < QMC_EVENTS of point q of replicate r takes its    */
/* holding-time word (word 0) from dimension 2k and its slot word (word 2)   */
/* from dimension 2k + 1; words 1 and 3 and all later events come from the   */
/* path's Philox block, with path index r 2^m + q.  Row b of L_(r,d) is word */
/* 0 of Philox counter {b, 0xFFFFFFFC, d, r} (bits above b kept, bit b set);  */
/* e_(i,r,d) is word d mod 4 of counter {d / 4, 0xFFFFFFFD, i, r}.            */
/* ------------------------------------------------------------------------ */
#define QMC_DIMS 16
#define QMC_EVENTS (QMC_DIMS / 2)
#define QMC_MAX_LOG2 24

static const struct {
    int s, a;
    uint32_t m[6];
} sobol_par[QMC_DIMS - 1] = {
    {1, 0, {1}},           {2, 1, {1, 3}},          {3, 1, {1, 3, 1}},         {3, 2, {1, 1, 1}},
    {4, 1, {1, 1, 3, 3}},  {4, 4, {1, 3, 5, 13}},   {5, 2, {1, 1, 5, 5, 17}},  {5, 4, {1, 1, 5, 5, 5}},
    {5, 7, {1, 1, 7, 11, 19}}, {5, 11, {1, 1, 5, 1, 1}}, {5, 13, {1, 1, 1, 3, 11}}, {5, 14, {1, 3, 5, 5, 31}},
    {6, 1, {1, 3, 3, 9, 7, 49}}, {6, 13, {1, 1, 1, 15, 21, 21}}, {6, 16, {1, 3, 1, 13, 27, 49}},
};

int oracle_qmc_dims(void) { return QMC_DIMS; }

/* Primitive-polynomial parameters of dimension d >= 1 (degree, coefficient bits). */
void oracle_sobol_poly(int d, int *s, int *a)
{
    *s = sobol_par[d - 1].s;
    *a = sobol_par[d - 1].a;
}

/* Unscrambled direction numbers V[d][b], d < QMC_DIMS, b < 32. */
void oracle_sobol_directions(uint32_t V[QMC_DIMS][32])
{
    for (int b = 0; b < 32; ++b) V[0][b] = 1u << (31 - b);
    for (int d = 1; d < QMC_DIMS; ++d) {
        int s = sobol_par[d - 1].s, a = sobol_par[d - 1].a;
        uint64_t m[33];
        for (int k = 1; k <= s; ++k) m[k] = sobol_par[d - 1].m[k - 1];
        for (int k = s + 1; k <= 32; ++k) {
            uint64_t x = (m[k - s] << s) ^ m[k - s];
            for (int c = 1; c < s; ++c)
                if ((a >> (s - 1 - c)) & 1) x ^= m[k - c] << c;
            m[k] = x;
        }
        for (int k = 1; k <= 32; ++k) V[d][k - 1] = (uint32_t)(m[k] << (32 - k));
    }
}

/* Coordinate of point q from 32 direction numbers. */
uint32_t oracle_sobol_point(const uint32_t *Vd, uint32_t q)
{
    uint32_t x = 0;
    for (int b = 0; q != 0; ++b, q >>= 1)
        if (q & 1u) x ^= Vd[b];
    return x;
}

static uint32_t parity32(uint32_t x)
{
    uint32_t p = 0;
    while (x) {
        p ^= 1u;
        x &= x - 1u;
    }
    return p;
}

/* Apply L_(r,d) to a 32-bit word. */
static uint32_t lms_apply(uint64_t seed, uint32_t r, uint32_t d, uint32_t x)
{
    uint32_t y = 0;
    for (uint32_t b = 0; b < 32; ++b) {
        uint32_t w[4];
        draw(seed, b, 0xFFFFFFFCu, ((uint64_t)r << 32) | d, w);
        uint32_t above = b == 0 ? 0u : (0xFFFFFFFFu << (32 - b));
        uint32_t row = (w[0] & above) | (1u << (31 - b));
        y |= parity32(row & x) << (31 - b);
    }
    return y;
}

/* Scrambled direction numbers of replicate r: out[d][b] = L_(r,d) V[d][b], b < 32. */
void oracle_qmc_scrambled(uint64_t seed, uint32_t r, uint32_t out[QMC_DIMS][32])
{
    uint32_t V[QMC_DIMS][32];
    oracle_sobol_directions(V);
    for (uint32_t d = 0; d < QMC_DIMS; ++d)
        for (int b = 0; b < 32; ++b) out[d][b] = lms_apply(seed, r, d, V[d][b]);
}

uint32_t oracle_qmc_shift(uint64_t seed, int32_t entry, uint32_t r, uint32_t d)
{
    uint32_t w[4];
    draw(seed, d / 4, 0xFFFFFFFDu, ((uint64_t)r << 32) | (uint32_t)entry, w);
    return w[d % 4];
}

typedef struct {
    const uint32_t (*V)[32]; /* scrambled direction numbers of the replicate */
    uint32_t e[QMC_DIMS];    /* digital shifts of (entry, replicate) */
    uint32_t q;              /* point index within the replicate */
} qmc_point;

static void qmc_override(const qmc_point *qp, uint32_t k, uint32_t w[4])
{
    if (k >= QMC_EVENTS) return;
    w[0] = oracle_sobol_point(qp->V[2 * k], qp->q) ^ qp->e[2 * k];
    w[2] = oracle_sobol_point(qp->V[2 * k + 1], qp->q) ^ qp->e[2 * k + 1];
}

/* ------------------------------------------------------------------------ */
/* One backward path (Algorithm 1 / Theorem 1, continuous-path reading).     */
/* ------------------------------------------------------------------------ */
typedef struct {
    int32_t end;
    uint32_t njumps;
    uint64_t hash;   /* FNV-1a 64 over the visited indices, start included */
    double logw;     /* log of the multiplicative functional */
} path_out;

#define FNV_OFFSET 14695981039346656037ull
#define FNV_PRIME 1099511628211ull

static int32_t pick_next(const oracle_graph *g, int32_t j, uint32_t w2, uint32_t w3)
{
    int64_t o = g->row_start[j];
    uint32_t slot = (uint32_t)(((uint64_t)w2 * (uint64_t)(uint32_t)g->deg[j]) >> 32);
    if (g->weighted[j] && !(w3 < g->thresh[o + slot])) return g->alias_col[o + slot];
    return g->edge_col[o + slot];
}

/* Grid points m*dt (m = 0..N-1) with m*dt <= rho, counted in the path's
 * remaining-time coordinate rho = t - time.  Single precision. */
static int grid_count_f32(float rho, float invdt, int N)
{
    if (rho < 0.0f) return 0;
    float f = floorf(rho * invdt);
    int c = (int)f + 1;
    return c < N ? c : N;
}

static int grid_count_f64(double rho, double invdt, int N)
{
    if (rho < 0.0) return 0;
    double f = floor(rho * invdt);
    int c = (int)f + 1;
    return c < N ? c : N;
}

static path_out path_f32(const oracle_graph *g, int32_t i, uint32_t stream, double t, int mode, int N, uint64_t seed, uint64_t p,
                         const qmc_point *qp)
{
    path_out o;
    int32_t j = i;
    float r = (float)t;
    float acc = 0.0f;
    float dt = (float)(t / (double)N);
    float invdt = (float)((double)N / t);
    uint32_t k = 0;
    uint64_t h = (FNV_OFFSET ^ (uint64_t)(uint32_t)i) * FNV_PRIME;
    for (;;) {
        float dl = g->delta32[j];
        if (g->deg[j] == 0) {
            if (mode == O_EXACT) acc = fmaf(dl, r, acc);
            else acc = fmaf(dl, (float)grid_count_f32(r, invdt, N), acc);
            break;
        }
        uint32_t w[4];
        draw(seed, k, stream, p, w);
        if (qp) qmc_override(qp, k, w);
        float S = -oracle_logf(unif_f32(w[0])) * g->inv_rate32[j];
        if (S >= r) {
            if (mode == O_EXACT) acc = fmaf(dl, r, acc);
            else acc = fmaf(dl, (float)grid_count_f32(r, invdt, N), acc);
            break;
        }
        float rn = r - S;
        if (mode == O_EXACT) acc = fmaf(dl, S, acc);
        else acc = fmaf(dl, (float)(grid_count_f32(r, invdt, N) - grid_count_f32(rn, invdt, N)), acc);
        r = rn;
        j = pick_next(g, j, w[2], w[3]);
        h = (h ^ (uint64_t)(uint32_t)j) * FNV_PRIME;
        ++k;
    }
    float logw;
    if (mode == O_EXACT) {
        logw = acc;
    } else if (mode == O_LIE) {
        logw = acc * dt;
    } else {
        float a = fmaf(0.5f, g->delta32[i], acc);
        a = fmaf(-0.5f, g->delta32[j], a);
        logw = a * dt;
    }
    o.end = j; o.njumps = k; o.hash = h; o.logw = (double)logw;
    return o;
}

static path_out path_f64(const oracle_graph *g, int32_t i, uint32_t stream, double t, int mode, int N, uint64_t seed, uint64_t p,
                         const qmc_point *qp)
{
    path_out o;
    int32_t j = i;
    double r = t;
    double acc = 0.0;
    double dt = t / (double)N;
    double invdt = (double)N / t;
    uint32_t k = 0;
    uint64_t h = (FNV_OFFSET ^ (uint64_t)(uint32_t)i) * FNV_PRIME;
    for (;;) {
        double dl = g->delta64[j];
        if (g->deg[j] == 0) {
            if (mode == O_EXACT) acc = fma(dl, r, acc);
            else acc = fma(dl, (double)grid_count_f64(r, invdt, N), acc);
            break;
        }
        uint32_t w[4];
        draw(seed, k, stream, p, w);
        if (qp) qmc_override(qp, k, w);
        double S = -oracle_log(unif_f64(w[0], w[1])) * g->inv_rate64[j];
        if (S >= r) {
            if (mode == O_EXACT) acc = fma(dl, r, acc);
            else acc = fma(dl, (double)grid_count_f64(r, invdt, N), acc);
            break;
        }
        double rn = r - S;
        if (mode == O_EXACT) acc = fma(dl, S, acc);
        else acc = fma(dl, (double)(grid_count_f64(r, invdt, N) - grid_count_f64(rn, invdt, N)), acc);
        r = rn;
        j = pick_next(g, j, w[2], w[3]);
        h = (h ^ (uint64_t)(uint32_t)j) * FNV_PRIME;
        ++k;
    }
    double logw;
    if (mode == O_EXACT) {
        logw = acc;
    } else if (mode == O_LIE) {
        logw = acc * dt;
    } else {
        double a = fma(0.5, g->delta64[i], acc);
        a = fma(-0.5, g->delta64[j], a);
        logw = a * dt;
    }
    o.end = j; o.njumps = k; o.hash = h; o.logw = logw;
    return o;
}

static path_out one_path_stream(const oracle_graph *g, int32_t i, uint32_t stream, double t, int mode,
                                int N, int prec, uint64_t seed, uint64_t p)
{
    if (t == 0.0) {  /* exp(0 A) v = v: no holding time, no weight */
        path_out o = {i, 0, (FNV_OFFSET ^ (uint64_t)(uint32_t)i) * FNV_PRIME, 0.0};
        return o;
    }
    return prec == 0 ? path_f32(g, i, stream, t, mode, N, seed, p, NULL) : path_f64(g, i, stream, t, mode, N, seed, p, NULL);
}

/* Backward paths of entry i draw from stream word i. */
static path_out one_path(const oracle_graph *g, int32_t i, double t, int mode, int N, int prec,
                         uint64_t seed, uint64_t p)
{
    return one_path_stream(g, i, (uint32_t)i, t, mode, N, prec, seed, p);
}

/* Per-path trace for parity checks: paths first_path .. first_path+count-1 of entry i. */
void oracle_trace(const oracle_graph *g, double t, int mode, int N, int prec, int32_t entry,
                  uint64_t seed, uint64_t first_path, uint32_t count,
                  int32_t *end, uint32_t *njumps, uint64_t *hash, double *logw)
{
    for (uint32_t q = 0; q < count; ++q) {
        path_out o = one_path(g, entry, t, mode, N, prec, seed, first_path + q);
        end[q] = o.end; njumps[q] = o.njumps; hash[q] = o.hash; logw[q] = o.logw;
    }
}

/* Sample mean of W v_{X_t} over paths path_offset .. path_offset+M-1 for each
 * requested entry (Algorithm 1 with the mean divided by M), with the standard
 * error sqrt(s^2 / M) where s^2 is the unbiased sample variance (Welford's
 * recurrence).  The mean itself is the plain sequential FP64 sum over paths
 * divided by M.  Entries run in parallel (OpenMP); each entry is sequential. */
int oracle_estimate(const oracle_graph *g, const double *v, double t, int mode, int N, int prec,
                    uint64_t M, const int32_t *entries, int64_t n_entries, uint64_t seed,
                    uint64_t path_offset, double *mean, double *sem, uint64_t *jumps_out)
{
    uint64_t jumps = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : jumps)
    for (int64_t q = 0; q < n_entries; ++q) {
        int32_t i = entries ? entries[q] : (int32_t)q;
        double sum = 0.0, wm = 0.0, wss = 0.0;
        for (uint64_t p = 0; p < M; ++p) {
            path_out o = one_path(g, i, t, mode, N, prec, seed, path_offset + p);
            double w = exp(o.logw) * v[o.end];
            sum += w;
            double d = w - wm;
            wm += d / (double)(p + 1);
            wss += d * (w - wm);
            jumps += o.njumps;
        }
        mean[q] = M ? sum / (double)M : 0.0;
        sem[q] = M > 1 ? sqrt(wss / (double)(M - 1) / (double)M) : 0.0;
    }
    if (jumps_out) *jumps_out = jumps;
    return O_OK;
}

/* Randomised QMC estimate: for each requested entry, replicates r0 .. r0+R-1 */
/* (R of them; disjoint ranges are independent and can be merged) of the      */
/* 2^log2q points of the scrambled Sobol' set (quasi-random draws for events */
/* 0..QMC_EVENTS-1, as described above); replicate mean mu_r = plain          */
/* sequential FP64 sum of W v_{X_t} over its points / 2^log2q; the estimate  */
/* is the mean of the mu_r and its standard error sqrt(s^2 / R) with s^2 the */
/* unbiased sample variance of the mu_r (two passes).  rep_means (nullable)   */
/* receives the mu_r, entry-major.                                            */
static void qmc_replicate(uint64_t seed, int32_t i, uint32_t r, uint32_t V[QMC_DIMS][32], qmc_point *qp)
{
    oracle_qmc_scrambled(seed, r, V);
    qp->V = (const uint32_t(*)[32])V;
    for (uint32_t d = 0; d < QMC_DIMS; ++d) qp->e[d] = oracle_qmc_shift(seed, i, r, d);
}

static path_out qmc_path(const oracle_graph *g, int32_t i, double t, int mode, int N, int prec, uint64_t seed,
                         uint32_t log2q, uint32_t r, const qmc_point *qp)
{
    uint64_t p = ((uint64_t)r << log2q) | qp->q;
    if (t == 0.0) {
        path_out o = {i, 0, (FNV_OFFSET ^ (uint64_t)(uint32_t)i) * FNV_PRIME, 0.0};
        return o;
    }
    return prec == 0 ? path_f32(g, i, (uint32_t)i, t, mode, N, seed, p, qp)
                     : path_f64(g, i, (uint32_t)i, t, mode, N, seed, p, qp);
}

int oracle_estimate_rqmc(const oracle_graph *g, const double *v, double t, int mode, int N, int prec,
                         uint32_t log2q, uint32_t R, uint32_t r0, const int32_t *entries, int64_t n_entries,
                         uint64_t seed, double *mean, double *sem, double *rep_means, uint64_t *jumps_out)
{
    if (log2q > QMC_MAX_LOG2 || R < 1) return O_E_INVALID;
    uint64_t jumps = 0;
    const uint32_t Q = 1u << log2q;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : jumps)
    for (int64_t e = 0; e < n_entries; ++e) {
        int32_t i = entries ? entries[e] : (int32_t)e;
        double *mu = (double *)malloc(sizeof(double) * R);
        uint32_t V[QMC_DIMS][32];
        for (uint32_t r = 0; r < R; ++r) {
            qmc_point qp;
            qmc_replicate(seed, i, r0 + r, V, &qp);
            double sum = 0.0;
            for (uint32_t q = 0; q < Q; ++q) {
                qp.q = q;
                path_out o = qmc_path(g, i, t, mode, N, prec, seed, log2q, r0 + r, &qp);
                sum += exp(o.logw) * v[o.end];
                jumps += o.njumps;
            }
            mu[r] = sum / (double)Q;
        }
        double m = 0.0;
        for (uint32_t r = 0; r < R; ++r) m += mu[r];
        m /= (double)R;
        double ss = 0.0;
        for (uint32_t r = 0; r < R; ++r) ss += (mu[r] - m) * (mu[r] - m);
        mean[e] = m;
        sem[e] = R > 1 ? sqrt(ss / (double)(R - 1) / (double)R) : 0.0;
        if (rep_means)
            for (uint32_t r = 0; r < R; ++r) rep_means[(uint64_t)e * R + r] = mu[r];
        free(mu);
    }
    if (jumps_out) *jumps_out = jumps;
    return O_OK;
}

/* Per-path trace of points q0 .. q0+count-1 of replicate r of entry i. */
void oracle_trace_rqmc(const oracle_graph *g, double t, int mode, int N, int prec, int32_t entry, uint64_t seed,
                       uint32_t log2q, uint32_t r, uint32_t q0, uint32_t count, int32_t *end, uint32_t *njumps,
                       uint64_t *hash, double *logw)
{
    uint32_t V[QMC_DIMS][32];
    qmc_point qp;
    qmc_replicate(seed, entry, r, V, &qp);
    for (uint32_t c = 0; c < count; ++c) {
        qp.q = q0 + c;
        path_out o = qmc_path(g, entry, t, mode, N, prec, seed, log2q, r, &qp);
        end[c] = o.end; njumps[c] = o.njumps; hash[c] = o.hash; logw[c] = o.logw;
    }
}

/* Multilevel Monte Carlo over the time step (Giles 2008) for the STRANG and  */
/* LIE functionals: the coupled level difference Y = v_{X_t} (W_{N} - W_{N/2})*/
/* evaluates both grids on the same path.  The draw schedule does not depend  */
/* on N, so the path is simply run twice with the same (seed, path) and N and  */
/* N/2 steps; E[Y] is the difference of the two split targets of Theorem 1.   */
/* Per-entry mean (plain sequential FP64 sum) and standard error (Welford).   */
int oracle_estimate_level_difference(const oracle_graph *g, const double *v, double t, int mode, int N, int prec,
                                     uint64_t M, const int32_t *entries, int64_t n_entries, uint64_t seed,
                                     uint64_t path_offset, double *mean, double *sem)
{
    if ((mode != O_STRANG && mode != O_LIE) || N < 2 || (N & 1)) return O_E_INVALID;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t q = 0; q < n_entries; ++q) {
        int32_t i = entries ? entries[q] : (int32_t)q;
        double sum = 0.0, wm = 0.0, wss = 0.0;
        for (uint64_t p = 0; p < M; ++p) {
            path_out f = one_path(g, i, t, mode, N, prec, seed, path_offset + p);
            path_out c = one_path(g, i, t, mode, N / 2, prec, seed, path_offset + p);
            double y = (exp(f.logw) - exp(c.logw)) * v[f.end];
            sum += y;
            double d = y - wm;
            wm += d / (double)(p + 1);
            wss += d * (y - wm);
        }
        mean[q] = M ? sum / (double)M : 0.0;
        sem[q] = M > 1 ? sqrt(wss / (double)(M - 1) / (double)M) : 0.0;
    }
    return O_OK;
}

/* ------------------------------------------------------------------------ */
/* Forward form (Lemma 2, Theorem 2; Algorithm 2), on the graph of B = A^T:  */
/* start j ~ v_j / V, walk B's rows with B's potential, deposit V W at the   */
/* end state.                                                                */
/*                                                                           */
/* The start draw is a two-level alias: the indices are cut into groups of   */
/* 1024 (the last one ragged); group g has sum S_g (sequential, index order) */
/* and V = sum of the S_g (sequential, group order).  A canonical Vose table */
/* over the S_g picks the group, a canonical Vose table over the group's v_j */
/* picks the member: P(j) = (S_g / V)(v_j / S_g) = v_j / V.  One Philox call */
/* {0, 0xFFFFFFFF, path}: w0/w1 pick the group, w2/w3 the member.  Walk      */
/* events use counter {k, 0xFFFFFFFE, path}.                                 */
/* ------------------------------------------------------------------------ */
#define START_GROUP 1024

int oracle_start_table(int64_t n, const double *v, int32_t *top_alias, uint32_t *top_thresh,
                       int32_t *in_alias, uint32_t *in_thresh, double *vsum_out)
{
    for (int64_t i = 0; i < n; ++i)
        if (!(v[i] >= 0.0) || !isfinite(v[i])) return O_E_INVALID;
    int64_t G = (n + START_GROUP - 1) / START_GROUP;
    double *S = (double *)malloc(sizeof(double) * (size_t)(G + 1));
    double V = 0.0;
    for (int64_t g = 0; g < G; ++g) {
        double s = 0.0;
        int64_t hi = (g + 1) * START_GROUP < n ? (g + 1) * START_GROUP : n;
        for (int64_t i = g * START_GROUP; i < hi; ++i) s += v[i];
        S[g] = s;
        V += s;
    }
    *vsum_out = V;
    if (!(V > 0.0)) {
        free(S);
        return O_E_INVALID;
    }
    int64_t m = G > START_GROUP ? G : START_GROUP;
    int32_t *ids = (int32_t *)malloc(sizeof(int32_t) * (size_t)m);
    double *q = (double *)malloc(sizeof(double) * (size_t)m);
    int *sm = (int *)malloc(sizeof(int) * (size_t)m);
    int *lg = (int *)malloc(sizeof(int) * (size_t)m);
    for (int64_t g = 0; g < G; ++g) ids[g] = (int32_t)g;
    vose_row((int)G, S, V, ids, top_alias, top_thresh, q, sm, lg);
    for (int64_t g = 0; g < G; ++g) {
        int64_t lo = g * START_GROUP;
        int d = (int)(((g + 1) * START_GROUP < n ? (g + 1) * START_GROUP : n) - lo);
        for (int k = 0; k < d; ++k) ids[k] = (int32_t)(lo + k);
        if (S[g] > 0.0) {
            vose_row(d, v + lo, S[g], ids, in_alias + lo, in_thresh + lo, q, sm, lg);
        } else {
            for (int k = 0; k < d; ++k) {
                in_alias[lo + k] = (int32_t)(lo + k);
                in_thresh[lo + k] = 0xFFFFFFFFu;
            }
        }
    }
    free(S); free(ids); free(q); free(sm); free(lg);
    return O_OK;
}

static int32_t forward_start(int64_t n, const int32_t *top_alias, const uint32_t *top_thresh,
                             const int32_t *in_alias, const uint32_t *in_thresh, uint64_t seed, uint64_t path)
{
    uint32_t w[4];
    draw(seed, 0u, 0xFFFFFFFFu, path, w);
    uint64_t G = (uint64_t)((n + START_GROUP - 1) / START_GROUP);
    int64_t g = (int64_t)(((uint64_t)w[0] * G) >> 32);
    if (!(w[1] < top_thresh[g])) g = top_alias[g];
    int64_t lo = g * START_GROUP;
    uint64_t d = (uint64_t)(((g + 1) * START_GROUP < n ? (g + 1) * START_GROUP : n) - lo);
    int64_t j = lo + (int64_t)(((uint64_t)w[2] * d) >> 32);
    if (!(w[3] < in_thresh[j])) j = in_alias[j];
    return (int32_t)j;
}

/* Per-state sums over paths path_offset .. path_offset+M-1 of Y = V W 1{X_t = i}
 * (sum1) and Y^2 (sum2).  Then x_i = sum1_i / M. */
void oracle_forward(const oracle_graph *g, int64_t n, const int32_t *top_alias, const uint32_t *top_thresh,
                    const int32_t *in_alias, const uint32_t *in_thresh, double V, double t, int mode, int N,
                    int prec, uint64_t M, uint64_t seed, uint64_t path_offset, double *sum1, double *sum2,
                    uint64_t *jumps_out)
{
    uint64_t jumps = 0;
    for (uint64_t p = 0; p < M; ++p) {
        uint64_t path = path_offset + p;
        int32_t j0 = forward_start(n, top_alias, top_thresh, in_alias, in_thresh, seed, path);
        path_out o = one_path_stream(g, j0, 0xFFFFFFFEu, t, mode, N, prec, seed, path);
        double w = V * exp(o.logw);
        sum1[o.end] += w;
        sum2[o.end] += w * w;
        jumps += o.njumps;
    }
    if (jumps_out) *jumps_out = jumps;
}

void oracle_forward_trace(const oracle_graph *g, int64_t n, const int32_t *top_alias, const uint32_t *top_thresh,
                          const int32_t *in_alias, const uint32_t *in_thresh, double t, int mode, int N, int prec,
                          uint64_t seed, uint64_t first_path, uint32_t count, int32_t *start, int32_t *end,
                          uint32_t *njumps, uint64_t *hash, double *logw)
{
    for (uint32_t q = 0; q < count; ++q) {
        uint64_t path = first_path + q;
        int32_t j0 = forward_start(n, top_alias, top_thresh, in_alias, in_thresh, seed, path);
        path_out o = one_path_stream(g, j0, 0xFFFFFFFEu, t, mode, N, prec, seed, path);
        start[q] = j0; end[q] = o.end; njumps[q] = o.njumps; hash[q] = o.hash; logw[q] = o.logw;
    }
}

/* ------------------------------------------------------------------------ */
/* Control-variate estimator (variance reduction, Sec. 5).  For any h with    */
/* h(0) = v, Duhamel's formula with the Feynman-Kac representation of        */
/* exp(sA) gives x_i = h(t, i) + E_i[ int_0^t W_s R(t - s, X_s) ds ] with    */
/* R = A h - dh/dtau.  For h(tau) = v + tau Av + tau^2 A^2v/2 + tau^3 c3,     */
/* R(tau, j) = a_j tau^2 + b_j tau^3 (a = A^3v/2 - 3 c3, b = A c3).  Over a   */
/* hold of length D in state j that starts with remaining time r and log     */
/* weight L, the integral is exactly                                         */
/*   e^L sum_k c_k D^{k+1} phi_k(delta_j D),  phi_k(z) = int_0^1 e^{zs} s^k ds */
/* with R(r - u) = c0 + c1 u + c2 u^2 + c3' u^3.  The path is the FP32 path  */
/* of the backward walker (same draws); the integral is evaluated in FP64.   */
/* ------------------------------------------------------------------------ */
double oracle_phi(int k, double z)
{
    if (fabs(z) <= 2.0) {
        /* series: sum_n z^n / (n! (n + k + 1)) */
        double term = 1.0, sum = 0.0;
        for (int n = 0; n < 40; ++n) {
            sum += term / (double)(n + k + 1);
            term *= z / (double)(n + 1);
        }
        return sum;
    }
    double ez = exp(z);
    double p = (ez - 1.0) / z;
    for (int m = 1; m <= k; ++m) p = (ez - (double)m * p) / z;
    return p;
}

static double hold_integral(double a, double b, double delta, double r, double D)
{
    double c0 = a * r * r + b * r * r * r;
    double c1 = -2.0 * a * r - 3.0 * b * r * r;
    double c2 = a + 3.0 * b * r;
    double c3 = -b;
    double z = delta * D;
    return c0 * D * oracle_phi(0, z) + c1 * D * D * oracle_phi(1, z) + c2 * D * D * D * oracle_phi(2, z) +
           c3 * D * D * D * D * oracle_phi(3, z);
}

/* Residual part of one path's control-variate estimate (FP32 path, EXACT functional). */
static double cv_path(const oracle_graph *g, int32_t i, double t, const double *ca, const double *cb, uint64_t seed,
                      uint64_t p, uint32_t *njumps)
{
    int32_t j = i;
    float r = (float)t;
    float L = 0.0f;
    double y = 0.0;
    uint32_t k = 0;
    for (;;) {
        float dl = g->delta32[j];
        if (g->deg[j] == 0) {
            y += exp((double)L) * hold_integral(ca[j], cb[j], (double)dl, (double)r, (double)r);
            break;
        }
        uint32_t w[4];
        draw(seed, k, (uint32_t)i, p, w);
        float S = -oracle_logf(unif_f32(w[0])) * g->inv_rate32[j];
        if (S >= r) {
            y += exp((double)L) * hold_integral(ca[j], cb[j], (double)dl, (double)r, (double)r);
            break;
        }
        y += exp((double)L) * hold_integral(ca[j], cb[j], (double)dl, (double)r, (double)S);
        L = fmaf(dl, S, L);
        r = r - S;
        j = pick_next(g, j, w[2], w[3]);
        ++k;
    }
    *njumps = k;
    return y;
}

/* Per-entry control-variate estimate: mean = h_i + mean of the residual
 * integrals, sem from the residual integrals' sample variance (Welford). */
int oracle_estimate_cv(const oracle_graph *g, const double *ca, const double *cb, const double *h, double t,
                       uint64_t M, const int32_t *entries, int64_t n_entries, uint64_t seed, uint64_t path_offset,
                       double *mean, double *sem)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t q = 0; q < n_entries; ++q) {
        int32_t i = entries ? entries[q] : (int32_t)q;
        double sum = 0.0, wm = 0.0, wss = 0.0;
        for (uint64_t p = 0; p < M; ++p) {
            uint32_t nj;
            double y = t == 0.0 ? 0.0 : cv_path(g, i, t, ca, cb, seed, path_offset + p, &nj);
            sum += y;
            double d = y - wm;
            wm += d / (double)(p + 1);
            wss += d * (y - wm);
        }
        mean[q] = h[i] + (M ? sum / (double)M : 0.0);
        sem[q] = M > 1 ? sqrt(wss / (double)(M - 1) / (double)M) : 0.0;
    }
    return O_OK;
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
