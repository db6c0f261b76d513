"""Pins for the control-variate oracle (oracle/cv.py and the CV estimator in walker.c).

* phi_k(z) = int_0^1 e^{zs} s^k ds against SciPy quadrature and closed forms.
* Zero variance when h is exact: for a 3-node directed path A^3 = 0, so
  exp(tA)v = v + tAv + t^2A^2v/2 and with c3 = 0 the residual R vanishes.
* Unbiasedness for an arbitrary (random) h: z-test against expm.
* The Taylor-only h already cuts the variance for short horizons.
* MLP gradients against central finite differences; BF16 rounding rule.
"""
import math

import numpy as np
import pytest

import workloads as W
import zstats
from oracle import cv as CV
from oracle import dense as OD
from oracle import walker as OW


@pytest.mark.parametrize("k", [0, 1, 2, 3])
@pytest.mark.parametrize("z", [-40.0, -3.0, -2.0, -0.7, -1e-4, 0.0, 1e-4, 0.9, 2.0, 2.5, 12.0, 40.0])
def test_phi_against_quadrature(k, z):
    quad = pytest.importorskip("scipy.integrate").quad
    want, err = quad(lambda s: math.exp(z * s) * s ** k, 0.0, 1.0, epsabs=1e-300, epsrel=2e-14, limit=200)
    assert abs(OW.phi(k, z) - want) <= 1e-13 * abs(want) + 1e-300


def test_phi_closed_forms():
    assert OW.phi(0, 0.0) == 1.0 and abs(OW.phi(3, 0.0) - 0.25) < 1e-16
    for z in (-5.0, 0.5, 3.0):
        assert abs(OW.phi(0, z) - math.expm1(z) / z) < 1e-14 * abs(math.expm1(z) / z)


def test_exact_h_gives_zero_variance():
    a = np.zeros((3, 3))
    a[0, 1] = 1.3
    a[1, 2] = 0.7  # strictly upper triangular: A^3 = 0
    csr = W.dense_to_csr(a)
    v = np.array([0.2, -1.0, 2.0])
    t = 0.9
    T = CV.taylor_terms(csr, v)
    assert np.allclose(np.linalg.matrix_power(a, 3), 0)
    exact = OD.expmv_dense(a, t, v)
    T2 = T[0] + t * T[1] + t * t * T[2] / 2
    assert np.allclose(T2, exact, rtol=1e-13)
    c3, ca, cb = CV.cv_coefficients(csr, T, t, T2)
    assert np.allclose(c3, 0) and np.allclose(ca, 0) and np.allclose(cb, 0)
    g = OW.Graph(csr)
    mean, sem = g.estimate_cv(ca, cb, T2, t, 5000, seed=1)
    assert np.allclose(mean, exact, rtol=1e-13) and np.all(sem == 0)


def _conditioned(n, seed, rate=1.5, dsd=1.0):
    rng = np.random.default_rng(seed)
    a = np.where(rng.random((n, n)) < 0.3, rng.lognormal(0, 1, (n, n)), 0.0)
    np.fill_diagonal(a, 0.0)
    a *= rate / a.sum(axis=1).mean()
    np.fill_diagonal(a, rng.normal(0, dsd, n) - a.sum(axis=1) + rng.normal(0, dsd, n))
    return a


def test_cv_unbiased_for_random_h():
    a = _conditioned(40, 21)
    csr = W.dense_to_csr(a)
    v = W.uniform_vector(40, 2, -1.0, 1.0)
    t = 0.8
    T = CV.taylor_terms(csr, v)
    xhat = np.random.default_rng(5).normal(0, 2.0, 40)  # an arbitrary (bad) prediction
    c3, ca, cb = CV.cv_coefficients(csr, T, t, xhat)
    g = OW.Graph(csr)
    mean, sem = g.estimate_cv(ca, cb, xhat, t, 20000, seed=3)
    zstats.check((mean - OD.expmv_dense(a, t, v)) / sem, samples=20000)


def test_taylor_only_h_reduces_variance():
    csr = W.erdos_renyi(400, 6, 2)
    v = W.uniform_vector(400, 1)
    lam = OD.power_iteration(csr.to_scipy())
    t = 0.5 / lam
    T = CV.taylor_terms(csr, v)
    T2 = T[0] + t * T[1] + t * t * T[2] / 2
    c3, ca, cb = CV.cv_coefficients(csr, T, t, T2)
    g = OW.Graph(csr)
    m_cv, s_cv = g.estimate_cv(ca, cb, T2, t, 2000, seed=4)
    m_pl, s_pl, _ = g.estimate(v, t, 2000, seed=4)
    x = OD.taylor_expmv(csr.to_scipy(), t, v)
    zstats.check((m_cv - x) / s_cv, samples=2000)
    assert np.median(s_pl / s_cv) > 10.0  # variance reduction by > 100x


def test_mlp_gradient_finite_differences():
    rng = np.random.default_rng(0)
    p = CV.init_params(3)
    X = rng.normal(size=(50, CV.N_FEATURES))
    tgt = rng.normal(size=50)
    loss, g = CV.loss_and_grad(p, X, tgt, round_weights=False)
    for name in ("W1", "b1", "W2", "b2", "W3", "b3"):
        q = {k: v.astype(np.float64) for k, v in p.items()}
        idx = tuple(rng.integers(0, s) for s in q[name].shape)
        h = 1e-6
        q[name][idx] += h
        lp, _ = CV.loss_and_grad(q, X, tgt, round_weights=False)
        q[name][idx] -= 2 * h
        lm, _ = CV.loss_and_grad(q, X, tgt, round_weights=False)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[name][idx]) <= 1e-6 * max(1.0, abs(fd)), name


def test_bf16_rounding():
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -2.5, 3.1415926], dtype=np.float32)
    y = CV.bf16(x)
    assert y[0] == 1.0 and y[1] == 1.0  # tie to even
    assert y[2] == np.float32(1.0 + 2 ** -7)
    assert y[3] == -2.5 and abs(y[4] - 3.140625) < 1e-7


def test_features_shapes_and_values():
    csr = W.erdos_renyi(300, 5, 1)
    v = W.uniform_vector(300, 3)
    F, T2, T = CV.features(csr, v, 0.05)
    assert F.shape == (300, 5) and np.all(np.isfinite(F))
    deg = np.diff(csr.row_ptr)
    assert np.allclose(F[:, 0], np.log1p(deg))
    assert np.allclose(T2, v + 0.05 * T[1] + 0.05 ** 2 * T[2] / 2)


def _fp32_bf16_forward(p, X, order=1):
    """A test-local evaluation inside the model the bound covers: FP32 first layer,
    one BF16 rounding of each hidden activation, FP32 sums in the given order."""
    Wb = {k: (CV.bf16(v) if k[0] == "W" else np.asarray(v, np.float32)) for k, v in p.items()}
    Xf = np.asarray(X, np.float32)
    z1 = Xf[:, ::order] @ Wb["W1"][::order] + Wb["b1"]
    h1 = CV.bf16(np.maximum(z1, 0).astype(np.float32))
    z2 = h1[:, ::order] @ Wb["W2"][::order] + Wb["b2"]
    h2 = np.maximum(z2, 0).astype(np.float32)
    return (h2[:, ::order] @ Wb["W3"][::order] + Wb["b3"])[:, 0].astype(np.float64)


def test_forward_error_bound_covers_bf16_hidden_and_fp32_sums():
    """The bound of one BF16 rounding per first-layer activation plus FP32 accumulation
    holds for FP32/BF16 evaluations in two summation orders, on several networks; the
    mean square of the difference in units of forward_rounding_sigma is 1 (to sampling
    error), while rounding toward zero instead of to nearest gives more than 2; a dropped
    bias, a transposed hidden weight or a missing ReLU exceeds the elementwise bound."""
    rng = np.random.default_rng(4)
    for seed in range(4):
        p = CV.init_params(seed)
        X = rng.normal(size=(1000, CV.N_FEATURES)).astype(np.float32).astype(np.float64)
        y, _ = CV.forward(p, X)
        bound = CV.forward_error_bound(p, X)
        sig = CV.forward_rounding_sigma(p, X)
        for order in (1, -1):
            d = _fp32_bf16_forward(p, X, order) - y
            assert np.all(np.abs(d) <= bound)
            assert 0.8 < np.mean((d / sig) ** 2) < 1.25
        # the same evaluation with the activations truncated to BF16 (round toward zero)
        Wb = {k: (CV.bf16(v) if k[0] == "W" else np.asarray(v, np.float32)) for k, v in p.items()}
        z1 = np.asarray(X, np.float32) @ Wb["W1"] + Wb["b1"]
        h1 = (np.maximum(z1, 0).astype(np.float32).view(np.uint32) & 0xFFFF0000).view(np.float32)
        yt = (np.maximum(h1 @ Wb["W2"] + Wb["b2"], 0) @ Wb["W3"] + Wb["b3"])[:, 0]
        assert np.mean(((yt - y) / sig) ** 2) > 2.0
        # plausible mistakes are detected
        q = dict(p, b2=np.zeros_like(p["b2"]))
        assert np.any(np.abs(_fp32_bf16_forward(q, X) - y) > bound)
        q = dict(p, W2=np.ascontiguousarray(p["W2"].T))
        assert np.any(np.abs(_fp32_bf16_forward(q, X) - y) > bound)
        Wb = {k: CV.bf16(v).astype(np.float64) if k[0] == "W" else v.astype(np.float64) for k, v in p.items()}
        no_relu = ((X @ Wb["W1"] + Wb["b1"]) @ Wb["W2"] + Wb["b2"]).clip(0) @ Wb["W3"] + Wb["b3"]
        assert np.any(np.abs(no_relu[:, 0] - y) > bound)


def _bf16_gradient_eval(p, X, target, rnd=CV.bf16, bug=None):
    """A test-local gradient evaluation inside the model the bound and the sigma cover:
    the forward pass of _fp32_bf16_forward, dy in FP32, the hidden backward signal
    d2 = dy W3^T [z2 > 0] rounded once by `rnd`, the sums in FP64 (below FP32's
    error).  `bug` plants a mistake: "d1_no_transpose" (d1 = d2 W2 instead of d2 W2^T),
    "no_mask2" (d2 without the z2 mask), "half_dy" (dy = (y - t) / B)."""
    Wb = {k: (CV.bf16(v) if k[0] == "W" else np.asarray(v, np.float32)) for k, v in p.items()}
    Xf = np.asarray(X, np.float32)
    z1 = Xf @ Wb["W1"] + Wb["b1"]
    h1 = rnd(np.maximum(z1, 0).astype(np.float32))
    z2 = (h1 @ Wb["W2"] + Wb["b2"]).astype(np.float32)
    h2 = np.maximum(z2, 0)
    y = (h2 @ Wb["W3"] + Wb["b3"])[:, 0]
    B = X.shape[0]
    dy = np.float32(1.0 if bug == "half_dy" else 2.0) * (y - np.asarray(target, np.float32)) * np.float32(1.0 / B)
    mask2 = np.ones_like(z2) if bug == "no_mask2" else (z2 > 0)
    d2 = rnd(np.where(mask2, dy[:, None] * Wb["W3"][:, 0][None, :], 0).astype(np.float32)).astype(np.float64)
    W2 = Wb["W2"].astype(np.float64)
    d1 = np.where(z1 > 0, d2 @ (W2 if bug == "d1_no_transpose" else W2.T), 0.0)
    h1, h2, dy = h1.astype(np.float64), h2.astype(np.float64), dy.astype(np.float64)
    return {"W1": np.asarray(X, np.float64).T @ d1, "b1": d1.sum(0), "W2": h1.T @ d2, "b2": d2.sum(0),
            "W3": (h2.T @ dy)[:, None], "b3": np.array([dy.sum()])}


def _truncate_bf16(a):
    return (np.asarray(a, np.float32).view(np.uint32) & 0xFFFF0000).view(np.float32)


def test_gradient_bound_and_sigma_cover_bf16_backward():
    """With h1 and the hidden backward signal rounded to BF16 (to nearest): every
    gradient entry within gradient_error_bound; the mean square of the differences in
    units of gradient_rounding_sigma near 1 (0.71 .. 1.56 over 20 networks of 777
    samples; here 8 networks must fall in [0.4, 3]), while truncation instead of
    rounding gives more than 10; a planted mistake (transposed W2 in the backward
    signal, a dropped ReLU mask, half the residual's factor) breaks the bound or the
    mean square."""
    rng = np.random.default_rng(9)
    for seed in range(8):
        p = CV.init_params(seed)
        X = rng.normal(size=(777, CV.N_FEATURES)).astype(np.float32).astype(np.float64)
        t = rng.normal(size=777)
        _, g = CV.loss_and_grad(p, X, t)
        bound, _ = CV.gradient_error_bound(p, X, t)
        sig = CV.gradient_rounding_sigma(p, X, t)

        def stats(h):
            inb = all(np.all(np.abs(h[k] - g[k]) <= bound[k]) for k in g)
            z = np.concatenate([((h[k] - g[k]) / sig[k]).ravel() for k in g])
            return inb, float(np.mean(z * z))

        inb, ms = stats(_bf16_gradient_eval(p, X, t))
        assert inb and 0.4 < ms < 3.0, (seed, ms)
        assert stats(_bf16_gradient_eval(p, X, t, rnd=_truncate_bf16))[1] > 10.0
        for bug in ("d1_no_transpose", "no_mask2", "half_dy"):
            inb, ms = stats(_bf16_gradient_eval(p, X, t, bug=bug))
            assert not inb or ms > 10.0, (seed, bug, ms)


def test_features_and_taylor_terms_brute_force():
    """Every feature column, the rates and the Taylor terms against per-node loops over
    explicit neighbour lists and dense matrix powers on a small weighted graph with a
    diagonal, a node without off-diagonal entries and a zero T2 (features divide by 1 there)."""
    rng = np.random.default_rng(11)
    n = 40
    a = np.where(rng.random((n, n)) < 0.15, rng.lognormal(0, 0.7, (n, n)), 0.0)
    a[5, :] = 0.0  # no positive off-diagonal entry: rate 0, no neighbours
    np.fill_diagonal(a, rng.normal(0, 1, n))
    csr = W.dense_to_csr(a)
    v = rng.uniform(-1, 1, n)
    v[5] = 0.0  # row 5 holds only its diagonal, so T2[5] = 0 exactly
    t = 0.37
    F, T2, T = CV.features(csr, v, t)
    for k in range(4):
        assert np.allclose(T[k], np.linalg.matrix_power(a, k) @ v, rtol=1e-12, atol=1e-13)
    lam = np.array([sum(a[i, j] for j in range(n) if j != i and a[i, j] > 0) for i in range(n)])
    assert np.allclose(CV.rates(csr)[0], lam, rtol=1e-14, atol=0)
    for i in range(n):
        nb = [lam[j] for j in range(n) if j != i and a[i, j] > 0]
        mean = float(np.mean(nb)) if nb else 0.0
        sd = float(np.sqrt(max(np.mean(np.square(nb)) - mean * mean, 0.0))) if nb else 0.0
        t2 = v[i] + t * T[1][i] + t * t * T[2][i] / 2
        t2s = t2 if t2 != 0 else 1.0
        want = [math.log1p(lam[i]), math.log1p(mean), math.log1p(sd), t * T[1][i] / t2s, t * t * T[2][i] / (2 * t2s)]
        assert np.allclose(F[i], want, rtol=1e-12, atol=1e-14), i
        assert abs(T2[i] - t2) <= 1e-14 * (abs(t2) + 1)
    assert T2[5] == 0.0 and np.all(F[5] == 0.0)


def test_training_targets():
    x = np.array([2.0, 1.0, -3.0, 1e-9, 5.0])
    T2 = np.array([1.0, 4.0, 1.0, 1.0, 5.0])
    y = CV.targets(x, T2)
    assert np.allclose(y[[0, 1, 4]], [math.log(2.0), math.log(0.25), 0.0], rtol=1e-15)
    assert y[2] == y[3] == math.log(1e-6)  # ratios clamped below at 1e-6


def test_cv_coefficients_are_the_residual_of_h():
    """For h(tau) = v + tau Av + tau^2 A^2 v/2 + c3 tau^3 with h(t) = xhat, the residual
    A h(tau) - h'(tau) is a tau^2 + b tau^3 (the source term of the control variate),
    checked with dense matrix powers and a central difference for h'."""
    rng = np.random.default_rng(4)
    n = 30
    a = np.where(rng.random((n, n)) < 0.2, rng.uniform(0.1, 1.0, (n, n)), 0.0)
    np.fill_diagonal(a, rng.normal(0, 0.5, n))
    csr = W.dense_to_csr(a)
    v = rng.uniform(0, 1, n)
    t = 0.6
    T = CV.taylor_terms(csr, v)
    xhat = rng.uniform(0.5, 2.0, n)
    c3, ca, cb = CV.cv_coefficients(csr, T, t, xhat)
    P = [np.linalg.matrix_power(a, k) @ v for k in range(3)]

    def h(tau):
        return P[0] + tau * P[1] + tau * tau * P[2] / 2 + c3 * tau ** 3

    assert np.allclose(h(t), xhat, rtol=1e-12)
    for tau in (0.1, 0.35, 0.6):
        eps = 1e-5
        dh = (h(tau + eps) - h(tau - eps)) / (2 * eps)
        r = a @ h(tau) - dh
        assert np.allclose(r, ca * tau ** 2 + cb * tau ** 3, rtol=1e-7, atol=1e-7 * np.abs(r).max())
