"""Learned control variate: features, MLP and coefficients in plain FP64 numpy
(test infrastructure only).

The estimator (variance reduction named in Sec. 5; written out in walker.c):
    x_i = h(t, i) + E_i[ int_0^t W_s R(t - s, X_s) ds ],  R = A h - dh/dtau,
unbiased for every h with h(0) = v.  Here
    h(tau) = v + tau Av + tau^2 A^2 v / 2 + tau^3 c3,
with c3 chosen so that h(t) equals the network's prediction xhat:
    c3 = (xhat - T2) / t^3,  T2 = v + t Av + t^2 A^2 v / 2,
so that R(tau) = a tau^2 + b tau^3, a = A^3 v / 2 - 3 c3, b = A c3.

The network: 5 node features -> 64 ReLU -> 64 ReLU -> 1, predicting
y = log(x / T2); xhat = T2 exp(y).  Weights are used rounded to BF16 (round to
nearest even), biases in full precision; everything else here is FP64.
`forward_error_bound` states how far an implementation of the same network
may land from this FP64 forward pass when it rounds each first-layer
activation to BF16 once and accumulates in FP32 (a bound from the arithmetic,
not a restatement of any implementation's operation order), and
`forward_rounding_sigma` the typical size of that difference when the
roundings are to nearest (independent errors, uniform over half an ulp).
"""
from __future__ import annotations

import numpy as np

N_FEATURES = 5
HIDDEN = 64


def _sp(csr):
    return csr.to_scipy()


def rates(csr):
    """lambda_i = sum of positive off-diagonal entries, deg_i = their count."""
    n = csr.n
    rows = np.repeat(np.arange(n), np.diff(csr.row_ptr))
    keep = (csr.col != rows) & (csr.val > 0)
    lam = np.bincount(rows[keep], weights=csr.val[keep], minlength=n)
    deg = np.bincount(rows[keep], minlength=n)
    return lam, deg, rows, keep


def taylor_terms(csr, v):
    """[v, Av, A^2 v, A^3 v] (A the full matrix, diagonal included)."""
    a = _sp(csr)
    t1 = a @ v
    t2 = a @ t1
    t3 = a @ t2
    return np.stack([np.asarray(v, dtype=np.float64), t1, t2, t3])


def features(csr, v, t):
    """Node features: log1p(lambda), log1p(mean neighbour lambda), log1p(std of
    neighbour lambda), t(Av)/T2, t^2(A^2v)/(2 T2); plus T2 and the Taylor terms."""
    lam, deg, rows, keep = rates(csr)
    cols = csr.col[keep]
    s1 = np.bincount(rows[keep], weights=lam[cols], minlength=csr.n)
    s2 = np.bincount(rows[keep], weights=lam[cols] ** 2, minlength=csr.n)
    dd = np.maximum(deg, 1)
    mean = np.where(deg > 0, s1 / dd, 0.0)
    var = np.maximum(np.where(deg > 0, s2 / dd - mean * mean, 0.0), 0.0)
    T = taylor_terms(csr, v)
    T2 = T[0] + t * T[1] + t * t * T[2] / 2.0
    T2s = np.where(T2 != 0.0, T2, 1.0)
    F = np.stack([np.log1p(lam), np.log1p(mean), np.log1p(np.sqrt(var)), t * T[1] / T2s,
                  t * t * T[2] / (2.0 * T2s)], axis=1)
    return F, T2, T


def targets(x, T2):
    """Training target y = log(x / T2) (ratio clamped below at 1e-6)."""
    return np.log(np.maximum(np.asarray(x) / T2, 1e-6))


def bf16(w):
    """Round FP32 values to BF16 (round to nearest, ties to even), returned as float32."""
    u = np.ascontiguousarray(w, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def init_params(seed: int = 0):
    rng = np.random.default_rng(seed)
    p = {}
    for name, (fi, fo) in (("1", (N_FEATURES, HIDDEN)), ("2", (HIDDEN, HIDDEN)), ("3", (HIDDEN, 1))):
        lim = np.sqrt(6.0 / fi)
        p["W" + name] = rng.uniform(-lim, lim, (fi, fo)).astype(np.float32)
        p["b" + name] = rng.uniform(-0.1, 0.1, fo).astype(np.float32)
    return p


def forward(p, X, round_weights=True):
    """MLP forward in FP64 (weights rounded to BF16 when round_weights); X standardised."""
    W = {k: (bf16(v) if (round_weights and k[0] == "W") else v).astype(np.float64) for k, v in p.items()}
    z1 = X @ W["W1"] + W["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W["W2"] + W["b2"]
    h2 = np.maximum(z2, 0.0)
    y = (h2 @ W["W3"] + W["b3"])[:, 0]
    return y, (X, z1, h1, z2, h2, W)


# unit roundoffs 2^-p of round to nearest: BF16 (p = 8 significand bits) and FP32 (p = 24)
U_BF16 = 2.0 ** -8
U_FP32 = 2.0 ** -24


def forward_error_bound(p, X):
    """Per-sample bound on |y' - y| between the FP64 forward pass y (BF16 weights) and
    any evaluation y' of the same network that
      - computes the first layer z1 in FP32 (6 terms: |e1| <= 2^-21 (|b1| + |X||W1|)),
      - rounds each ReLU(z1) to BF16 once (relative error <= 2^-8),
      - accumulates the 64 -> 64 layer in FP32 in any order, allowing a non-IEEE
        accumulator (taken as 2^-16 of the sum of magnitudes, 4x the IEEE bound 64 u),
      - accumulates the 64 -> 1 output layer in FP32 (65 terms: <= 2^-17.9).
    ReLU is 1-Lipschitz, so errors propagate through |W2| and |W3|.  Standard
    forward-error analysis (Higham, Accuracy and Stability of Numerical
    Algorithms, 2nd ed., Sec. 3.1: |fl(sum) - sum| <= gamma_k sum |terms|)."""
    y, (X, z1, h1, z2, h2, W) = forward(p, X, round_weights=True)
    A1, A2, A3 = np.abs(W["W1"]), np.abs(W["W2"]), np.abs(W["W3"])
    e1 = 2.0 ** -21 * (np.abs(W["b1"]) + np.abs(X) @ A1)            # FP32 first layer
    dh1 = (1.0 + U_BF16) * e1 + U_BF16 * np.abs(h1)                 # + one BF16 rounding
    dz2 = dh1 @ A2 + 2.0 ** -16 * ((np.abs(h1) + dh1) @ A2 + np.abs(W["b2"]))
    dy = (dz2 @ A3)[:, 0] + 2.0 ** -17 * (np.abs(W["b3"][0]) + ((np.abs(h2) + dz2) @ A3)[:, 0])
    return dy + 1e-12


def forward_rounding_sigma(p, X):
    """Standard deviation of the output change when every first-layer activation h1_k is
    rounded to the nearest BF16 value, the errors taken as independent and uniform over
    half an ulp (ulp = 2^(floor(log2 h1_k) - 7), variance ulp^2 / 12), to first order:
    dy = sum_k dh1_k g_k with g_k = dy/dh1_k = sum_j W2_kj [z2_j > 0] W3_j."""
    y, (X, z1, h1, z2, h2, W) = forward(p, X, round_weights=True)
    g = (W["W2"][None, :, :] * (z2 > 0)[:, None, :] * W["W3"][:, 0][None, None, :]).sum(-1)
    pos = h1 > 0
    ulp = np.where(pos, np.exp2(np.floor(np.log2(np.where(pos, h1, 1.0))) - 7), 0.0)
    return np.sqrt(((ulp * g) ** 2).sum(1) / 12.0) + 1e-12


def loss_and_grad(p, X, target, round_weights=True):
    """Mean squared error and its gradient (with respect to the weights as used)."""
    y, (X, z1, h1, z2, h2, W) = forward(p, X, round_weights)
    B = X.shape[0]
    r = y - target
    loss = float(np.mean(r * r))
    dy = (2.0 / B) * r[:, None]
    g = {"W3": h2.T @ dy, "b3": dy.sum(axis=0)}
    d2 = (dy @ W["W3"].T) * (z2 > 0)
    g["W2"] = h1.T @ d2
    g["b2"] = d2.sum(axis=0)
    d1 = (d2 @ W["W2"].T) * (z1 > 0)
    g["W1"] = X.T @ d1
    g["b1"] = d1.sum(axis=0)
    return loss, g


def cv_coefficients(csr, T, t, xhat):
    """c3 = (xhat - T2)/t^3, a = A^3 v/2 - 3 c3, b = A c3."""
    T2 = T[0] + t * T[1] + t * t * T[2] / 2.0
    c3 = (np.asarray(xhat, dtype=np.float64) - T2) / t ** 3
    a = T[3] / 2.0 - 3.0 * c3
    b = _sp(csr) @ c3
    return c3, a, b
