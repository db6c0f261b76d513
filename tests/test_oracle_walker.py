"""Pins for the C oracle walker (oracle/walker.c).

The walker is random, so it is pinned by: published known-answer vectors
(Philox), library routines it must agree with (log), exact structural facts
(rates, potentials, alias-table probabilities), invariants that hold path by
path (zero potential, constant potential, diagonal A), laws that hold in
distribution (Poisson jump counts, jump probabilities k_ij), and statistical
agreement with the independently pinned FP64 references of oracle/dense.py.
"""
import math
import os

import numpy as np
import pytest

import workloads as W
import zstats
from oracle import dense as OD
from oracle import walker as OW

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _z_ok(mean, sem, x, samples):
    """Per-entry z-scores z = (mean - x)/sem over k entries: the three bounds of
    tests/zstats.py (tail fraction, mean, and the variance when samples >= 1000)."""
    return zstats.check((mean - x) / sem, samples=samples)


# ---------------------------------------------------------------------------
# Philox4x32-10 and the logarithm
# ---------------------------------------------------------------------------

def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLD, "philox4x32_10_kat.txt")) if l.strip() and l[0] != "#"]
    assert len(rows) == 3
    for r in rows:
        vals = [int(x, 16) for x in r]
        out = OW.philox4x32_10(vals[:4], vals[4:6])
        assert [int(x) for x in out] == vals[6:10]


def test_philox_words_uniform():
    """All four words are uniform in their top bits over consecutive counters."""
    outs = np.array([OW.philox4x32_10([k, 7, 3, 0], [11, 0]) for k in range(4000)], dtype=np.uint64)
    for w in range(4):
        hist = np.bincount((outs[:, w] >> 28).astype(int), minlength=16)
        chi2 = float(((hist - 250.0) ** 2 / 250.0).sum())
        assert chi2 < 50.0  # 15 dof, p ~ 1e-5


def test_own_logf_against_libm():
    rng = np.random.default_rng(1)
    xs = np.concatenate([rng.uniform(0, 1, 20000), 2.0 ** -rng.uniform(0, 24, 5000), [2.0 ** -24, 0.5, 1.0],
                         rng.uniform(1, 1e6, 5000), 2.0 ** rng.uniform(-126, 127, 5000)])
    xs = xs.astype(np.float32)
    xs = xs[xs > 0]
    got = OW.logf_many(xs).astype(np.float64)
    want = np.log(xs.astype(np.float64))
    ulp = np.where(want != 0, np.spacing(np.abs(want).astype(np.float32)).astype(np.float64), 1e-45)
    assert np.all(np.abs(got - want) <= 2 * ulp + 1e-45)
    assert OW.logf(1.0) == 0.0


def test_own_logf_exhaustive_on_the_walker_uniforms():
    """Every uniform the FP32 walker can draw, u = K 2^-24 for K = 1 .. 2^24: the
    logarithm is within 2 ulp of the correctly rounded value (FP64 log rounded), never
    positive, exactly 0 only at u = 1, and monotone non-decreasing in u (so a larger
    uniform never gives a longer holding time)."""
    K = np.arange(1, 2 ** 24 + 1, dtype=np.float64)
    u = (K * 2.0 ** -24).astype(np.float32)
    got = OW.logf_many(u).astype(np.float64)
    want = np.log(u.astype(np.float64))
    ulp = np.where(want != 0, np.spacing(np.abs(want).astype(np.float32)).astype(np.float64), 1e-45)
    err = np.abs(got - want) / ulp
    assert err.max() <= 2.0, (err.max(), u[np.argmax(err)])
    assert np.all(got <= 0) and got[-1] == 0.0 and np.all(got[:-1] < 0)
    assert np.all(np.diff(got) >= 0)


def test_own_logf_table_against_its_definition():
    """Row j of the breakpoint table: 1/c_j rounded to FP32 for c_j = 1 + j/64, and
    -ln(1/c_j) (j <= 26) or -ln(2/c_j) (j >= 27) of that rounded value, rounded to
    FP32, checked with 40-digit decimal logarithms (so no row sits on a rounding tie
    of the FP64 logarithm the oracle takes)."""
    from decimal import Decimal, getcontext

    getcontext().prec = 40
    inv, L = OW.ln_table()
    for j in range(65):
        assert inv[j] == np.float32(1.0 / (1.0 + j / 64.0))
        a = Decimal(float(inv[j])) * (2 if j >= 27 else 1)
        assert L[j] == np.float32(float(-a.ln())), j
    assert inv[0] == 1.0 and L[0] == 0.0 and inv[64] == 0.5 and L[64] == 0.0
    assert np.all(np.abs(L) <= np.float32(math.log(2) / 2 + 0.01))


def test_own_log_against_libm():
    rng = np.random.default_rng(2)
    xs = np.concatenate([rng.uniform(0, 1, 20000), 2.0 ** -rng.uniform(0, 53, 5000), [2.0 ** -53, 0.5]])
    for x in xs[::7]:
        got = OW.log(float(x))
        want = math.log(float(x))
        assert abs(got - want) <= 2 * np.spacing(abs(want)), (x, got, want)
    assert OW.log(1.0) == 0.0


# ---------------------------------------------------------------------------
# Preparation (A = D - L, Sec. 2) and jump tables (Sec. 4)
# ---------------------------------------------------------------------------

def _conditioned_matrix(n, seed, rate=1.5, dsd=1.0):
    """Weighted non-symmetric A with mean jump rate `rate` and potentials spread
    by about `dsd`, so that path weights stay moderate and z-tests are sharp."""
    rng = np.random.default_rng(seed)
    a = np.where(rng.random((n, n)) < 0.3, rng.lognormal(0, 1, (n, n)), 0.0)
    np.fill_diagonal(a, 0.0)
    a *= rate / a.sum(axis=1).mean()
    np.fill_diagonal(a, rng.normal(0, dsd, n) - a.sum(axis=1) + rng.normal(0, dsd, n))
    return a


def _random_matrix(n, seed, weighted=True, neg_diag=True):
    rng = np.random.default_rng(seed)
    a = np.where(rng.random((n, n)) < 0.3, rng.lognormal(0, 1, (n, n)) if weighted else 1.0, 0.0)
    np.fill_diagonal(a, rng.normal(0, 2, n) if neg_diag else 0.0)
    return a


def test_prep_rates_and_potentials():
    a = _random_matrix(40, 0)
    a[3, :] = 0.0
    a[3, 3] = -1.5  # isolated node: lambda = 0
    g = OW.Graph(W.dense_to_csr(a))
    assert g.status == 0
    off = a - np.diag(np.diag(a))
    lam = off.sum(axis=1)
    assert np.array_equal(g.deg, (off > 0).sum(axis=1))
    assert np.allclose(g.delta64, np.diag(a) + lam, rtol=1e-15, atol=1e-15)
    nz = lam > 0
    assert np.allclose(g.inv_rate64[nz], 1.0 / lam[nz], rtol=1e-15)
    assert np.array_equal(g.inv_rate32, g.inv_rate64.astype(np.float32))
    assert np.array_equal(g.delta32, g.delta64.astype(np.float32))
    assert g.deg[3] == 0
    assert np.array_equal(g.row_start, np.concatenate([[0], np.cumsum(g.deg)[:-1]]))


def test_prep_uniform_rows_detected():
    g = OW.Graph(W.erdos_renyi(200, 5, 1))
    assert g.weighted.sum() == 0
    g = OW.Graph(W.dense_to_csr(_random_matrix(30, 1)))
    assert g.weighted[g.deg > 1].all()


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_alias_tables_reproduce_jump_probabilities(seed):
    """Each slot keeps its own column with probability thresh/2^32 and the alias
    otherwise; summed over slots this must give k_ij = a_ij / lambda_i (Eq. paths)."""
    a = _random_matrix(50, seed)
    g = OW.Graph(W.dense_to_csr(a))
    for i in range(50):
        d = int(g.deg[i])
        if d == 0:
            continue
        o = int(g.row_start[i])
        prob = np.zeros(50)
        for k in range(d):
            p_keep = (float(g.thresh[o + k]) / 2.0 ** 32) if g.weighted[i] else 1.0
            if g.thresh[o + k] == 0xFFFFFFFF:
                p_keep = 1.0
            prob[g.edge_col[o + k]] += p_keep / d
            prob[g.alias_col[o + k]] += (1.0 - p_keep) / d
        off = a[i].copy()
        off[i] = 0.0
        want = off / off.sum()
        assert np.abs(prob - want).max() <= d * 2.0 ** -32 + 1e-15


@pytest.mark.parametrize("bad", ["unsorted", "range", "negoff", "nan"])
def test_prep_rejects_invalid(bad):
    a = W.dense_to_csr(_random_matrix(10, 3))
    col, val = a.col.copy(), a.val.copy()
    r0, r1 = int(a.row_ptr[2]), int(a.row_ptr[3])
    if bad == "unsorted":
        col[r0], col[r0 + 1] = col[r0 + 1], col[r0]
        want = -1
    elif bad == "range":
        col[r1 - 1] = 10
        want = -1
    elif bad == "negoff":
        k = [p for p in range(r0, r1) if col[p] != 2][0]
        val[k] = -0.5
        want = -2
    else:
        val[r0] = float("nan")
        want = -3
    g = OW.Graph(W.CSR(10, a.row_ptr, col, val))
    assert g.status == want


# ---------------------------------------------------------------------------
# Path-level invariants
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_zero_potential_unit_vector_gives_exactly_one(prec):
    """delta = 0 (a CTMC generator) and v = 1: every path has W = 1, so every estimate is 1.0."""
    q = W.random_generator(100, 3)
    g = OW.Graph(q)
    assert np.abs(g.delta64).max() < 1e-12
    # make the potential exactly zero by building A with diag = -sum(off) in exact arithmetic
    tr = g.trace(1.0, 5, 0, 0, 50, prec=prec)
    assert np.abs(tr["logw"]).max() < 1e-10
    for mode in ("exact", "strang", "lie"):
        m, s, _ = g.estimate(np.ones(100), 0.7, 64, entries=np.arange(0, 100, 9), mode=mode, nsteps=4, prec=prec)
        assert np.abs(m - 1.0).max() < 1e-9


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_constant_potential_gives_constant_weight(prec):
    """Cycle adjacency: delta = 2 everywhere, so logW = 2t on every path in every mode."""
    n = 16
    a = np.zeros((n, n))
    for i in range(n):
        a[i, (i + 1) % n] = a[i, (i - 1) % n] = 1.0
    g = OW.Graph(W.dense_to_csr(a))
    t = 1.3
    tol = 1e-5 if prec == "fp32" else 1e-13
    for mode in ("exact", "strang", "lie"):
        tr = g.trace(t, 4, 9, 0, 200, mode=mode, nsteps=8, prec=prec)
        assert np.abs(tr["logw"] - 2.0 * t).max() < tol * 2.0 * t
        assert tr["njumps"].mean() > 1.0


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_diagonal_matrix_is_exact(prec):
    d = np.array([-2.0, 0.0, 0.3, 1.7])
    g = OW.Graph(W.dense_to_csr(np.diag(d)))
    v = np.array([1.0, 2.0, -3.0, 0.5])
    m, s, jumps = g.estimate(v, 0.9, 10, prec=prec)
    assert jumps == 0
    tol = 1e-6 if prec == "fp32" else 1e-15
    assert np.abs(m - np.exp(0.9 * d) * v).max() <= tol * np.abs(np.exp(0.9 * d) * v).max()
    assert np.all(s == 0.0)


def test_zero_time_returns_v():
    g = OW.Graph(W.erdos_renyi(50, 4, 0))
    v = W.uniform_vector(50, 1)
    m, s, jumps = g.estimate(v, 0.0, 5)
    assert np.allclose(m, v, rtol=4e-16, atol=0) and jumps == 0  # (v+...+v)/M rounds


def test_trace_deterministic_and_seed_dependent():
    g = OW.Graph(W.erdos_renyi(500, 8, 2))
    a = g.trace(0.5, 7, 123, 1000, 64)
    b = g.trace(0.5, 7, 123, 1000, 64)
    c = g.trace(0.5, 7, 124, 1000, 64)
    assert all(np.array_equal(a[k], b[k]) for k in a)
    assert not np.array_equal(a["hash"], c["hash"])
    # the index sequence does not depend on the functional or its quadrature
    d = g.trace(0.5, 7, 123, 1000, 64, mode="strang", nsteps=5)
    assert np.array_equal(a["hash"], d["hash"]) and np.array_equal(a["end"], d["end"])


# ---------------------------------------------------------------------------
# Laws of the sampler (Sec. 3, Eq. paths)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_jump_counts_poisson_on_regular_graph(prec):
    """On a k-regular graph the rate is k everywhere, so N_t ~ Poisson(k t)."""
    n, kdeg, t = 64, 4, 0.75
    a = np.zeros((n, n))
    for i in range(n):
        for s in (1, 2):
            a[i, (i + s) % n] = a[i, (i - s) % n] = 1.0
    g = OW.Graph(W.dense_to_csr(a))
    tr = g.trace(t, 0, 5, 0, 40000, prec=prec)
    lam = kdeg * t
    counts = np.bincount(tr["njumps"].astype(int), minlength=12)[:12].astype(float)
    probs = np.array([math.exp(-lam) * lam ** k / math.factorial(k) for k in range(12)])
    exp_c = probs * tr["njumps"].size
    keep = exp_c > 5
    chi2 = float(((counts[keep] - exp_c[keep]) ** 2 / exp_c[keep]).sum())
    assert chi2 < 35.0, chi2  # ~8 dof


def test_first_jump_distribution_weighted_row():
    """P(exactly one jump, X_t = j) = a_ij (e^{-lam_j t} - e^{-lam_i t}) / (lam_i - lam_j):
    a jump at time s ~ lam_i e^{-lam_i s} to j with probability k_ij (Eq. paths), then
    no jump from j in the remaining t - s."""
    a = _random_matrix(12, 5)
    g = OW.Graph(W.dense_to_csr(a))
    i = int(np.argmax(g.deg))
    off = a - np.diag(np.diag(a))
    lam = off.sum(axis=1)
    t = 0.3 / lam[i]
    P = 200000
    tr = g.trace(t, i, 1, 0, P)
    one = tr["end"][tr["njumps"] == 1]
    counts = np.bincount(one, minlength=12).astype(float)
    want = np.zeros(12)
    for j in range(12):
        if off[i, j] > 0:
            want[j] = off[i, j] * (math.exp(-lam[j] * t) - math.exp(-lam[i] * t)) / (lam[i] - lam[j])
    want *= P
    keep = want > 5
    chi2 = float(((counts[keep] - want[keep]) ** 2 / want[keep]).sum())
    assert chi2 < 3 * keep.sum() + 20, chi2
    # no-jump probability is e^{-lambda t}
    p0 = float((tr["njumps"] == 0).mean())
    assert abs(p0 - math.exp(-0.3)) < 5 * math.sqrt(p0 * (1 - p0) / P)


# ---------------------------------------------------------------------------
# Statistical agreement with exp(tA)v and the split products (Thm 1, Thm 2)
# ---------------------------------------------------------------------------

def test_backward_full_vector_vs_expm_weighted_mixed_potential():
    a = _conditioned_matrix(60, 7)
    t = 1.0
    v = W.uniform_vector(60, 3, -1.0, 1.0)
    x = OD.expmv_dense(a, t, v)
    g = OW.Graph(W.dense_to_csr(a))
    for prec in ("fp32", "fp64"):
        m, s, _ = g.estimate(v, t, 4000, seed=1, prec=prec)
        _z_ok(m, s, x, 4000)


def test_backward_grid2d_vs_kronecker():
    m_ = 16
    a = W.grid_laplacian_2d(m_)
    t = 10.0 / (4 * (m_ + 1) ** 2)
    v = W.uniform_vector(m_ * m_, 0)
    x = OD.grid2d_expmv(m_, t, v)
    g = OW.Graph(a)
    mean, sem, _ = g.estimate(v, t, 2000, seed=2)
    _z_ok(mean, sem, x, 2000)


@pytest.mark.parametrize("kind", ["strang", "lie"])
def test_split_modes_vs_split_products(kind):
    """STRANG(N) / LIE(N) are unbiased for the split products x^S / x^L (Theorem 1,
    Eqs. eq_general1 and deff).  N = 2 makes the split error far larger than the
    statistical error, so a mode that estimated exp(tA)v, or the other split,
    fails the test."""
    a = _conditioned_matrix(30, 9)
    t, N = 2.0, 2
    v = W.uniform_vector(30, 4, 0.2, 1.0)
    g = OW.Graph(W.dense_to_csr(a))
    xs = OD.split_expmv(a, t, N, v, kind)
    other = OD.split_expmv(a, t, N, v, "lie" if kind == "strang" else "strang")
    exact = OD.expmv_dense(a, t, v)
    m, s, _ = g.estimate(v, t, 20000, seed=3, mode=kind, nsteps=N, prec="fp64")
    _z_ok(m, s, xs, 20000)
    assert np.abs((m - other) / s).max() > 6
    assert np.abs((m - exact) / s).max() > 6


def test_forward_full_vector_nonsymmetric():
    """Theorem 2 on a non-symmetric A: walk the rows of B = A^T from j ~ v/V."""
    a = _conditioned_matrix(25, 11)
    t = 1.0
    v = W.uniform_vector(25, 5, 0.0, 1.0)
    x = OD.expmv_dense(a, t, v)
    gb = OW.Graph(W.dense_to_csr(a.T))
    mean, sem, _ = gb.forward(v, t, 400000, seed=4, prec="fp64")
    _z_ok(mean, sem, x, 400000 // 25)
    # walking A's own rows instead (a transposed operand) is visibly wrong
    ga = OW.Graph(W.dense_to_csr(a))
    bad, bsem, _ = ga.forward(v, t, 400000, seed=4, prec="fp64")
    assert np.abs((bad - x) / bsem).max() > 6


def test_forward_ctmc_transient_conserves_probability():
    q = W.random_generator(80, 2)
    p0 = W.dirichlet_probability(80, 3)
    g = OW.Graph(q)  # forward on B = Q estimates exp(t Q^T) p0
    want = OD.expmv_dense(q.to_dense().T, 1.0, p0)
    x, sem, _ = g.forward(p0, 1.0, 200000, seed=1)
    assert abs(x.sum() - 1.0) < 1e-9  # every path deposits V W = 1 somewhere
    _z_ok(x[sem > 0], sem[sem > 0], want[sem > 0], 200000 // 80)


def test_standard_error_matches_spread_and_sqrt_m_law():
    """The reported SE matches the spread across independent seeds and falls as
    M^-1/2 (Sec. 5)."""
    g = OW.Graph(W.erdos_renyi(100, 5, 4))
    v = np.ones(100)
    ent = np.array([3, 50])
    sp = {}
    for M in (250, 4000):
        means = np.array([g.estimate(v, 0.4, M, entries=ent, seed=s)[0] for s in range(40)])
        sems = np.array([g.estimate(v, 0.4, M, entries=ent, seed=s)[1] for s in range(3)])
        sp[M] = means.std(axis=0, ddof=1)
        assert np.all(np.abs(sp[M] / sems.mean(axis=0) - 1.0) < 0.4)
    ratio = sp[250] / sp[4000]
    assert np.all((ratio > 2.6) & (ratio < 6.0))  # sqrt(16) = 4


def test_path_offset_splits_compose():
    g = OW.Graph(W.erdos_renyi(100, 5, 4))
    v = W.uniform_vector(100, 0)
    ent = np.arange(0, 100, 7)
    m_all, _, _ = g.estimate(v, 0.5, 300, entries=ent, seed=8)
    m_a, _, _ = g.estimate(v, 0.5, 100, entries=ent, seed=8, path_offset=0)
    m_b, _, _ = g.estimate(v, 0.5, 200, entries=ent, seed=8, path_offset=100)
    assert np.allclose((100 * m_a + 200 * m_b) / 300, m_all, rtol=1e-13, atol=0)


def test_forward_start_tables_reproduce_v():
    """The two-level start table (group of 1024, then member) implies P(j) = v_j / V
    (Lemma 2) up to the 2^-32 threshold quantisation; zero entries are never drawn."""
    n, GS = 2500, OW.START_GROUP
    rng = np.random.default_rng(3)
    v = rng.exponential(1.0, n)
    v[rng.random(n) < 0.2] = 0.0
    v[1024:2048] = 0.0  # an all-zero group
    g = OW.Graph(W.dense_to_csr(np.eye(n)))
    st, t = g.start_table(v)
    assert st == 0
    G = (n + GS - 1) // GS

    def implied(alias, thresh, d):
        p = np.zeros(d)
        for k in range(d):
            keep = 1.0 if thresh[k] == 0xFFFFFFFF else thresh[k] / 2.0 ** 32
            p[k] += keep / d
            p[alias[k]] += (1.0 - keep) / d
        return p

    pg = implied(t["top_alias"], t["top_thresh"], G)
    P = np.zeros(n)
    for gi in range(G):
        lo, hi = gi * GS, min(n, (gi + 1) * GS)
        if pg[gi] == 0:
            continue
        pin = implied(t["in_alias"][lo:hi] - lo, t["in_thresh"][lo:hi], hi - lo)
        P[lo:hi] = pg[gi] * pin
    assert abs(t["V"] - v.sum()) <= 1e-12 * v.sum()
    assert np.abs(P - v / v.sum()).max() <= (G + GS) * 2.0 ** -32
    assert np.all(P[v == 0] == 0)
    tr = g.forward_trace(v, 0.0, 5, 0, 20000)
    assert np.all(v[tr["start"]] > 0)


def test_total_communicability_from_forward_paths():
    """TC(t) = 1^T exp(tA) 1 = n E[W] over the forward paths of v = 1 (Theorem 2 with
    v = 1, Sec. 6), for EXACT and the split products (1^T S 1 for S the Strang or
    Lie product: the scalar is the same for S and its transpose)."""
    csr = W.erdos_renyi(200, 5, 2)
    a = csr.to_scipy().toarray()
    g = OW.Graph(csr)
    t, N, M = 0.3, 2, 200000
    for mode in ("exact", "strang", "lie"):
        x = OD.expmv_dense(a, t, np.ones(200)) if mode == "exact" else OD.split_expmv(a, t, N, np.ones(200), mode)
        want = float(x.sum())
        tr = g.forward_trace(np.ones(200), t, 7, 0, M, mode=mode, nsteps=N, prec="fp64")
        w = np.exp(tr["logw"])
        z = (200 * w.mean() - want) / (200 * w.std(ddof=1) / np.sqrt(M))
        assert abs(z) < 4, (mode, z)
