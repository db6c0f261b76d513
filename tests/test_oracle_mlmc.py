"""Pins of the oracle's multilevel level-difference estimator (coupled STRANG/LIE
functionals at N and N/2 steps on the same paths):

* a diagonal matrix (no jumps) gives W_N = W_{N/2} on every path, so every
  difference is exactly zero;
* the coupling telescopes: the plain estimate at N_0 plus the level differences
  at N_1 .. N_L, all on the same paths, equals the plain estimate at N_L to FP64
  rounding (a mis-coupled level, e.g. another path or a wrong coarse grid, fails);
* the mean matches the difference of the dense split products of Theorem 1
  (z-scores), for STRANG and LIE;
* the per-path variance of a level falls by about 4 per level (log-log slope
  about -2 in N: the pathwise quadrature error of a piecewise-constant potential
  is O(dt) for both rules).
"""
import math

import numpy as np
import pytest

import workloads as W
import zstats
from oracle import dense as OD
from oracle import walker as OW


def _graph():
    rng = np.random.default_rng(5)
    n = 40
    a = np.where(rng.random((n, n)) < 0.15, rng.uniform(0.2, 1.5, (n, n)), 0.0)
    np.fill_diagonal(a, rng.normal(0, 1, n))
    return W.dense_to_csr(a), a


def test_no_jumps_zero_difference():
    a = np.diag(np.linspace(-1.0, 2.0, 12))
    csr = W.dense_to_csr(a)
    g = OW.Graph(csr)
    v = W.uniform_vector(12, 3)
    for mode in ("strang", "lie"):
        m, s = g.estimate_level_difference(v, 0.7, 8, 200, mode=mode)
        assert np.all(m == 0.0) and np.all(s == 0.0)


@pytest.mark.parametrize("mode", ["strang", "lie"])
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_levels_telescope_on_the_same_paths(mode, prec):
    csr, _ = _graph()
    g = OW.Graph(csr)
    v = W.uniform_vector(csr.n, 1, -1.0, 1.0)
    t, M, off = 0.9, 3000, 12345
    n0, L = 2, 4
    base, _, _ = g.estimate(v, t, M, seed=7, path_offset=off, mode=mode, nsteps=n0, prec=prec)
    total = base.copy()
    for lvl in range(1, L + 1):
        d, _ = g.estimate_level_difference(v, t, n0 << lvl, M, seed=7, path_offset=off, mode=mode, prec=prec)
        total += d
    fine, _, _ = g.estimate(v, t, M, seed=7, path_offset=off, mode=mode, nsteps=n0 << L, prec=prec)
    scale, _, _ = g.estimate(np.abs(v), t, M, seed=7, path_offset=off, mode=mode, nsteps=n0 << L, prec=prec)
    assert np.all(np.abs(total - fine) <= 1e-12 * scale), np.max(np.abs(total - fine) / scale)


@pytest.mark.parametrize("mode", ["strang", "lie"])
def test_level_mean_matches_split_products(mode):
    csr, a = _graph()
    g = OW.Graph(csr)
    v = W.uniform_vector(csr.n, 2)
    t, N = 0.9, 4
    exact = OD.split_expmv(a, t, N, v, mode) - OD.split_expmv(a, t, N // 2, v, mode)
    m, s = g.estimate_level_difference(v, t, N, 40000, seed=11, mode=mode, prec="fp64")
    zstats.check((m - exact) / s, samples=40000)


def test_level_variance_decay():
    """Per-path variance of the level difference against N = 16 .. 128: log-log
    slope about -2 (variance O(dt^2))."""
    csr, _ = _graph()
    g = OW.Graph(csr)
    v = np.ones(csr.n)
    M = 40000
    Ns = (16, 32, 64, 128)
    for mode in ("strang", "lie"):
        V = []
        for N in Ns:
            _, s = g.estimate_level_difference(v, 0.9, N, M, seed=3, mode=mode, prec="fp64")
            V.append(np.mean(s ** 2) * M)
        slope = np.polyfit(np.log(Ns), np.log(V), 1)[0]
        assert -2.5 < slope < -1.5, (mode, slope)
