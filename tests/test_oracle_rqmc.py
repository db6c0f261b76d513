"""Pins of the oracle's randomised quasi-Monte Carlo estimator (variance reduction,
Sec. 5) against facts fixed by the mathematics of Sobol' nets and by the exact
exp(tA)v:

* every polynomial is primitive over GF(2) (the multiplicative order of x modulo
  it is 2^s - 1, by brute force) and every initial m_k is odd and below 2^k;
* dimension 0 is van der Corput's sequence (bit reversal of the index), and the
  first points of dimension 1 are the ones worked out by hand from x + 1, m_1 = 1;
* the first 2^m points are a (t, m, s)-net with t = sum of (degree - 1) over the
  dimensions (every elementary box of volume 2^(t-m) holds exactly 2^t points),
  before and after the random linear scramble and digital shift, which must both
  keep the net (an upper-triangular or otherwise wrong scramble breaks it);
* the estimator is unbiased (z-scores against expm over many entries), its
  standard error matches the spread of independent replicate sets, and it has a
  smaller variance than plain Monte Carlo with as many paths;
* the first holding times of one replicate are stratified: the number of points
  with no jump in [0, t) differs from 2^m e^{-lambda t} by at most one.
"""
import itertools
import math

import numpy as np
import pytest
import scipy.linalg

import workloads as W
import zstats
from oracle import dense as OD
from oracle import walker as OW


def _poly_order(s, a):
    """Multiplicative order of x modulo p(x) = x^s + a_1 x^(s-1) + ... + a_(s-1) x + 1 (bits)."""
    p = (1 << s) | 1
    for c in range(1, s):
        if (a >> (s - 1 - c)) & 1:
            p |= 1 << (s - c)
    x, k = 2 % p if s > 1 else 1, 1  # x mod p (for s = 1, x = 1 mod x + 1)
    while x != 1:
        x <<= 1
        if x >> s & 1:
            x ^= p
        k += 1
        assert k < 1 << s
    return k


def test_polynomials_primitive_and_initial_numbers():
    V = OW.sobol_directions()
    for d in range(1, OW.qmc_dims()):
        s, a = OW.sobol_poly(d)
        assert _poly_order(s, a) == (1 << s) - 1, d
        for k in range(1, 33):  # m_k = V[k-1] >> (32 - k) is odd and below 2^k
            m = int(V[d, k - 1]) >> (32 - k)
            assert m & 1 and m < (1 << k) and (int(V[d, k - 1]) & ((1 << (32 - k)) - 1)) == 0, (d, k)
    # distinct polynomials (a repeated one would repeat a dimension's generator matrix)
    assert len({OW.sobol_poly(d) for d in range(1, OW.qmc_dims())}) == OW.qmc_dims() - 1


def test_first_dimensions_by_hand():
    P = OW.sobol_points(OW.sobol_directions(), 64)
    rev = [int(f"{q:032b}"[::-1], 2) for q in range(64)]
    assert list(P[:, 0]) == rev
    # x + 1, m_1 = 1: m = 1, 3, 5, 15 -> v = 1/2, 3/4, 5/8, 15/16
    assert list(P[:8, 1] / 2.0 ** 32) == [0, 0.5, 0.75, 0.25, 0.625, 0.125, 0.375, 0.875]


def _is_net(P, dims, m, t):
    """(t, m, s)-net check of the first 2^m points over the given dimensions."""
    X = P[: 1 << m][:, dims].astype(np.uint64)
    for ks in itertools.product(range(m - t + 1), repeat=len(dims)):
        if sum(ks) != m - t:
            continue
        key = np.zeros(X.shape[0], np.uint64)
        for j, k in enumerate(ks):
            key = (key << np.uint64(k)) | (X[:, j] >> np.uint64(32 - k) if k else np.uint64(0))
        counts = np.bincount(key.astype(np.int64), minlength=1 << (m - t))
        if not np.all(counts == (1 << t)):
            return False
    return True


def _t_value(dims):
    return sum(max(OW.sobol_poly(d)[0] - 1, 0) if d else 0 for d in dims)


@pytest.mark.parametrize("dims", [(0, 1), (0, 1, 2), (2, 3), (0, 1, 2, 3, 4), (6, 7), (14, 15)])
def test_net_property_plain_and_scrambled(dims):
    t = _t_value(dims)
    m = max(10, t + 4)
    base = OW.sobol_points(OW.sobol_directions(), 1 << m)
    assert _is_net(base, list(dims), m, t)
    for r in range(3):
        Vs = OW.qmc_scrambled(seed=5, replicate=r)
        P = OW.sobol_points(Vs, 1 << m)
        sh = np.array([OW.qmc_shift(5, 17, r, d) for d in range(OW.qmc_dims())], np.uint32)
        assert _is_net(P ^ sh, list(dims), m, t)
        assert not np.array_equal(P, base)  # the scramble is not the identity


def test_net_check_detects_a_wrong_scramble():
    """The net check is sensitive to the scramble's orientation: a matrix that
    mixes less significant bits into more significant ones (upper-triangular)
    breaks the two-dimensional net of dimensions 0 and 1."""
    m = 8
    P = OW.sobol_points(OW.sobol_directions(), 1 << m)[:, :2]
    rng = np.random.default_rng(0)
    Y = np.zeros(P.shape, np.uint64)
    for d in range(2):
        rows = [(int(rng.integers(0, 1 << 32)) & ((1 << (31 - b)) - 1)) | (1 << (31 - b)) for b in range(32)]
        Y[:, d] = [sum((bin(int(xv) & rw).count("1") & 1) << (31 - b) for b, rw in enumerate(rows)) for xv in P[:, d]]
    assert _is_net(P, [0, 1], m, 0) and not _is_net(Y, [0, 1], m, 0)


def _small_graph():
    csr = W.erdos_renyi(60, 4, 3)
    a = csr.to_scipy().toarray()
    return csr, a


def test_rqmc_unbiased_against_expm():
    csr, a = _small_graph()
    t = 0.35
    v = W.uniform_vector(csr.n, 1)
    x = scipy.linalg.expm(t * a) @ v
    g = OW.Graph(csr)
    # the standard error comes from 16 replicate means: z ~ Student t with 15 dof
    mean, sem, _ = g.estimate_rqmc(v, t, 6, 16, seed=3)
    zstats.check((mean - x) / sem, samples=16, dof=15)
    # FP64 paths and a split functional: unbiased for their own targets
    mean64, sem64, _ = g.estimate_rqmc(v, t, 6, 16, seed=4, prec="fp64")
    zstats.check((mean64 - x) / sem64, samples=16, dof=15)
    xs = OD.split_expmv(a, t, 2, v, "strang")
    ms, ss, _ = g.estimate_rqmc(v, t, 6, 16, seed=6, mode="strang", nsteps=2)
    zstats.check((ms - xs) / ss, samples=16, dof=15)


def test_rqmc_standard_error_and_variance_reduction():
    csr, a = _small_graph()
    t = 0.35
    v = np.ones(csr.n)
    x = scipy.linalg.expm(t * a) @ v
    g = OW.Graph(csr)
    ent = np.arange(8, dtype=np.int32)
    runs = [g.estimate_rqmc(v, t, 7, 8, entries=ent, seed=s) for s in range(24)]
    means = np.array([r[0] for r in runs])
    sems = np.array([r[1] for r in runs])
    spread = means.std(axis=0, ddof=1)
    ratio = np.sqrt((sems ** 2).mean(axis=0)) / spread
    assert np.all((ratio > 0.6) & (ratio < 1.6)), ratio
    assert np.all(np.abs(means.mean(axis=0) - x[ent]) < 4 * spread / math.sqrt(len(runs)) + 1e-12)
    # plain Monte Carlo with the same 8 * 2^7 paths per entry
    mc = np.array([g.estimate(v, t, 8 << 7, entries=ent, seed=100 + s)[0] for s in range(24)])
    var_ratio = (means.var(axis=0, ddof=1) / mc.var(axis=0, ddof=1)).mean()
    assert var_ratio < 0.5, var_ratio


def test_first_holding_times_stratified():
    """2^m points of one replicate: the count of paths with no jump before t
    (first uniform u <= e^{-lambda t}) is within one of 2^m e^{-lambda t}."""
    csr, _ = _small_graph()
    g = OW.Graph(csr)
    t = 0.2
    for i in (0, 5, 11):
        lam = float(np.float32(1.0) / g.inv_rate32[i])
        for r in range(3):
            tr = g.trace_rqmc(t, i, 9, 8, r, 0, 256)
            zero = int(np.sum(tr["njumps"] == 0))
            assert abs(zero - 256 * math.exp(-lam * t)) <= 1.0 + 1e-3, (i, r, zero)


def test_one_point_replicates_are_plain_monte_carlo():
    """log2_points = 0: every replicate is one uniformly shifted point, i.e. an
    independent Monte Carlo path; the estimate is still unbiased."""
    csr, a = _small_graph()
    t = 0.35
    v = W.uniform_vector(csr.n, 2)
    x = scipy.linalg.expm(t * a) @ v
    mean, sem, reps = OW.Graph(csr).estimate_rqmc(v, t, 0, 256, seed=8)
    assert reps.shape == (csr.n, 256)
    zstats.check((mean - x) / sem, samples=256, dof=255)


def test_replicate_ranges_merge_like_one_run():
    """Two disjoint replicate ranges (two ranks) merged by the shard formula give the
    single run over all replicates: the same replicate means, the same estimate and
    standard error."""
    from paper_1904_12759_gb300 import shard

    csr, _ = _small_graph()
    g = OW.Graph(csr)
    v = W.uniform_vector(csr.n, 5)
    m, s, reps = g.estimate_rqmc(v, 0.3, 5, 12, seed=21)
    m1, s1, r1 = g.estimate_rqmc(v, 0.3, 5, 7, seed=21)
    m2, s2, r2 = g.estimate_rqmc(v, 0.3, 5, 5, seed=21, replicate_offset=7)
    assert np.array_equal(np.concatenate([r1, r2], axis=1), reps)
    mm, ss = shard.merge(np.stack([m1, m2]), np.stack([s1, s2]), np.array([7, 5]))
    # the merge's one-pass variance leaves ~1e-8 of the mean where the spread is zero
    assert np.allclose(mm, m, rtol=1e-13, atol=0)
    assert np.allclose(ss, s, rtol=1e-8, atol=1e-7 * np.abs(m).max())


def test_rqmc_unbiased_on_weighted_rows():
    """Alias rows: the quasi-random slot word picks the table slot, Philox word 3 the
    alias acceptance; the estimate stays unbiased (z-scores against expm) and keeps a
    smaller spread than plain Monte Carlo with as many paths."""
    rng = np.random.default_rng(17)
    n = 50
    a = np.where(rng.random((n, n)) < 0.2, rng.lognormal(0.0, 1.0, (n, n)), 0.0)
    np.fill_diagonal(a, rng.normal(0.0, 0.5, n))
    csr = W.dense_to_csr(a)
    g = OW.Graph(csr)
    assert g.weighted.any()
    t = 0.3
    v = W.uniform_vector(n, 9)
    x = scipy.linalg.expm(t * a) @ v
    mean, sem, _ = g.estimate_rqmc(v, t, 6, 16, seed=12)
    zstats.check((mean - x) / sem, samples=16, dof=15)
    _, sem_mc, _ = g.estimate(v, t, 16 << 6, seed=12)
    assert np.mean(sem ** 2) < np.mean(sem_mc ** 2)


def test_first_event_jointly_stratified_on_a_star():
    """Entry 0 of a star with four absorbing leaves (rate 4, t = ln 2 / 4): a path
    jumps iff its first holding word falls in the half [0, 1/2) of dimension 0, and
    its leaf is the quarter of dimension 1 its slot word falls in.  Dimensions 0 and
    1 form a (0, m, 2)-net (kept by the scramble and the shift), so each box
    [0, 1/2) x [k/4, (k+1)/4) holds exactly 2^m / 8 of a replicate's points: half
    the paths jump and each leaf receives exactly an eighth, with no sampling noise."""
    a = np.zeros((5, 5))
    a[0, 1:] = 1.0
    csr = W.dense_to_csr(a)
    g = OW.Graph(csr)
    t = math.log(2.0) / 4.0
    m = 8
    for r in range(4):
        tr = g.trace_rqmc(t, 0, 31, m, r, 0, 1 << m)
        jumped = tr["njumps"] == 1
        assert int(jumped.sum()) == (1 << m) // 2, r
        counts = np.bincount(tr["end"][jumped], minlength=5)[1:]
        assert np.all(counts == (1 << m) // 8), (r, counts)
    # the same number of plain Monte Carlo paths is not stratified (sensitivity of the check)
    tp = g.trace(t, 0, 31, 0, 1 << m)
    plain = np.bincount(tp["end"][tp["njumps"] == 1], minlength=5)[1:]
    assert not np.all(plain == (1 << m) // 8)
