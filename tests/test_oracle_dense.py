"""Pins for the deterministic FP64 references in oracle/dense.py.

Each check compares against something other than the oracle itself: a closed
form, a mathematical invariant, an independent method, or SciPy.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import dense as OD


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def test_expm_diagonal():
    d = np.array([-3.0, 0.0, 0.5, 2.0, 7.5])
    assert rel(np.diag(OD.expm_dense(np.diag(d))), np.exp(d)) < 1e-14


def test_expm_2x2_symmetric_closed_form():
    a, b, t = 0.7, -1.3, 2.1
    m = np.array([[a, b], [b, a]])
    e = math.exp(t * a)
    want = e * np.array([[math.cosh(t * b), math.sinh(t * b)], [math.sinh(t * b), math.cosh(t * b)]])
    assert rel(OD.expm_dense(t * m), want) < 1e-14


def test_two_state_ctmc_closed_form():
    al, be, t = 2.0, 0.5, 0.9
    q = np.array([[-al, al], [be, -be]])
    s = al + be
    e = math.exp(-s * t)
    want = np.array([[be + al * e, al - al * e], [be - be * e, al + be * e]]) / s
    assert rel(OD.expm_dense(t * q), want) < 1e-14
    v = np.array([0.3, -1.2])
    assert rel(OD.uniformization_expmv(q, t, v), want @ v) < 1e-13
    assert rel(OD.taylor_expmv(q, t, v), want @ v) < 1e-13


@pytest.mark.parametrize("n", [5, 8, 13])
def test_cycle_graph_circulant(n):
    beta = 0.8
    a = np.zeros((n, n))
    for i in range(n):
        a[i, (i + 1) % n] = a[i, (i - 1) % n] = 1.0
    m = np.arange(n)
    lam = 2.0 * np.cos(2.0 * np.pi * m / n)
    want = np.empty((n, n))
    for j in range(n):
        for k in range(n):
            want[j, k] = np.mean(np.exp(beta * lam) * np.cos(2.0 * np.pi * m * (j - k) / n))
    assert rel(OD.expm_dense(beta * a), want) < 1e-13


def test_complete_graph_total_communicability():
    n, beta = 9, 0.37
    a = np.ones((n, n)) - np.eye(n)
    want = np.full(n, math.exp(beta * (n - 1)))
    assert rel(OD.expmv_dense(a, beta, np.ones(n)), want) < 1e-13
    assert rel(OD.taylor_expmv(W.dense_to_csr(a).to_scipy(), beta, np.ones(n)), want) < 1e-13


def test_grid2d_kronecker_vs_dense_vs_taylor():
    m = 6
    a = W.grid_laplacian_2d(m)
    t = 3.0 / a.to_dense().diagonal().__abs__().max() * 4
    v = W.uniform_vector(m * m, 3)
    x_k = OD.grid2d_expmv(m, t, v)
    x_d = OD.expmv_dense(a.to_dense(), t, v)
    x_t = OD.taylor_expmv(a.to_scipy(), t, v)
    assert rel(x_k, x_d) < 1e-12
    assert rel(x_t, x_d) < 1e-12


def test_grid3d_kronecker_vs_dense_and_rows():
    m = 4
    a = W.grid_laplacian_3d(m)
    t = 0.01
    v = W.uniform_vector(m ** 3, 4)
    x_k = OD.grid3d_expmv(m, t, v)
    x_d = OD.expmv_dense(a.to_dense(), t, v)
    assert rel(x_k, x_d) < 1e-12
    rows = np.array([0, 5, 17, 63])
    assert rel(OD.grid3d_expmv(m, t, v, rows=rows), x_d[rows]) < 1e-12


def test_uniformization_vs_dense_and_conservation():
    q = W.random_generator(60, 5)
    qd = q.to_dense()
    assert np.abs(qd.sum(axis=1)).max() < 1e-12
    p0 = W.dirichlet_probability(60, 1)
    for t in (0.1, 1.0, 10.0):
        x_u = OD.uniformization_expmv(q.to_scipy(), t, np.ones(60))
        assert np.abs(x_u - 1.0).max() < 1e-13  # exp(tQ) 1 = 1
        # transient p(t)^T = p0^T exp(tQ)  <=>  p(t) = exp(t Q^T) p0
        pt_d = OD.expmv_dense(qd.T, t, p0)
        pt_u = OD.uniformization_expmv(q.to_scipy().T.tocsr(), t, p0)
        assert rel(pt_u, pt_d) < 1e-12
        assert abs(pt_d.sum() - 1.0) < 1e-12
        assert rel(OD.taylor_expmv(q.to_scipy().T.tocsr(), t, p0), pt_d) < 1e-12


def test_scipy_expm_cross_check():
    sl = pytest.importorskip("scipy.linalg")
    rng = np.random.default_rng(7)
    a = rng.standard_normal((30, 30))
    a = (a + a.T) / 2
    assert rel(OD.expm_dense(a), sl.expm(a)) < 1e-11


def _two_state_split_by_hand(a11, a12, a22, t, N, v, kind):
    """Split product for a 2x2 symmetric A, with e^{-dt L} from the 2-state closed form."""
    lam = a12
    d = np.array([a11 + a12, a22 + a12])
    dt = t / N
    e = math.exp(-2.0 * lam * dt)
    p = 0.5 * np.array([[1 + e, 1 - e], [1 - e, 1 + e]])
    x = np.array(v, dtype=float)
    for _ in range(N):
        if kind == "lie":
            x = p @ (np.exp(dt * d) * x)
        else:
            x = np.exp(0.5 * dt * d) * (p @ (np.exp(0.5 * dt * d) * x))
    return x


@pytest.mark.parametrize("kind", ["lie", "strang"])
def test_split_products_two_state_by_hand(kind):
    a = np.array([[-1.0, 0.8], [0.8, 2.5]])
    v = np.array([1.3, -0.4])
    got = OD.split_expmv(a, 1.7, 3, v, kind)
    want = _two_state_split_by_hand(-1.0, 0.8, 2.5, 1.7, 3, v, kind)
    assert rel(got, want) < 1e-13


def test_split_orders_and_tc_superconvergence():
    """Lie is O(dt), Strang O(dt^2) per entry; for TC = 1^T x both are O(dt^2) (Sec. 5)."""
    g = W.erdos_renyi(40, 4, 11)
    a = g.to_dense()
    t = 0.5
    x = OD.expmv_dense(a, t, np.ones(40))
    v = np.ones(40)
    errs = {}
    for kind in ("lie", "strang"):
        e_entry, e_tc = [], []
        for N in (8, 16, 32):
            xs = OD.split_expmv(a, t, N, v, kind)
            e_entry.append(np.abs(xs - x).max())
            e_tc.append(abs(xs.sum() - x.sum()))
        errs[kind] = (e_entry, e_tc)
    le, ltc = errs["lie"]
    se, stc = errs["strang"]
    assert 1.7 < le[0] / le[1] < 2.3 and 1.7 < le[1] / le[2] < 2.3  # first order per entry
    assert 3.5 < se[0] / se[1] < 4.5 and 3.5 < se[1] / se[2] < 4.5  # second order
    assert 3.5 < ltc[0] / ltc[1] < 4.5  # Lie gains an order on TC since L 1 = 0
    # error bound of Sec. 5 on TC: |(1, D L D 1)| dt^2 per unit time, bounded by 2 d_max^3 dt^2
    dmax = a.sum(axis=1).max()
    dt = t / 32
    assert stc[2] <= 2 * dmax ** 3 * dt ** 2 * x.sum()


def test_split_exact_when_potential_constant():
    """Regular graph: D = d I commutes with L, so both splits are exact."""
    n = 12
    a = np.zeros((n, n))
    for i in range(n):
        a[i, (i + 1) % n] = a[i, (i - 1) % n] = 1.0
    v = W.uniform_vector(n, 2)
    x = OD.expmv_dense(a, 0.9, v)
    for kind in ("lie", "strang"):
        assert rel(OD.split_expmv(a, 0.9, 2, v, kind), x) < 1e-13


def test_power_iteration():
    n = 10
    k = np.ones((n, n)) - np.eye(n)
    assert abs(OD.power_iteration(k) - (n - 1)) < 1e-10
    g = W.erdos_renyi(300, 6, 3).to_scipy()
    want = float(np.linalg.eigvalsh(g.toarray()).max())
    assert abs(OD.power_iteration(g, iters=20000, tol=1e-14) - want) / want < 1e-8
