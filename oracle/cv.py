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
roundings are to nearest (independent errors, uniform over half an ulp);
`gradient_error_bound` does the same for the gradient of the squared error when
the backward signal of the hidden layer is rounded to BF16 once too.
"""
from __future__ import annotations

import numpy as np
from scipy.special import erfc

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


def gradient_error_bound(p, X, target, tile=128):
    """Elementwise bounds on |g' - g| and |loss' - loss| between the FP64 gradient g of
    `loss_and_grad` (BF16 weights) and any evaluation g' that
      - runs the forward pass as `forward_error_bound` allows (FP32 first layer, each
        ReLU(z1) rounded to BF16 once, FP32 sums), so |z2' - z2| <= dz2 and |y' - y| <= dyv;
      - forms dy = 2 (y - target) / B in FP32 and the hidden backward signal
        d2 = dy W3^T [z2 > 0], rounded to BF16 once (relative <= 2^-8);
      - forms d1 = d2 W2^T (64 terms) and dW2 = h1^T d2, db2 = sum d2 over tiles of
        `tile` samples with FP32 accumulation in any order (taken as 4x the IEEE
        bound: 2^-16 of the sum of magnitudes for 64 terms, 2^-15 for 128), the tiles
        then summed in FP32 (one more 2^-24 per tile);
      - forms dW1 = X^T d1 [z1 > 0], db1, dW3 = h2^T dy, db3 and the loss in FP32 over
        the tiles ((tile + tiles) 2^-24 of the sums of magnitudes).
    A ReLU mask may differ where |z| is within its forward error of zero: such units
    contribute their whole magnitude.  Errors propagate through |W2| and |W3| (ReLU is
    1-Lipschitz); standard forward-error analysis (Higham, Sec. 3.1)."""
    y, (X, z1, h1, z2, h2, W) = forward(p, X, round_weights=True)
    B = X.shape[0]
    nb = -(-B // tile)
    u = U_BF16
    A2, A3 = np.abs(W["W2"]), np.abs(W["W3"])
    w3 = W["W3"][:, 0]
    e1 = 2.0 ** -21 * (np.abs(W["b1"]) + np.abs(X) @ np.abs(W["W1"]))
    Dh1 = (1.0 + u) * e1 + u * np.abs(h1)
    dz2 = Dh1 @ A2 + 2.0 ** -16 * ((np.abs(h1) + Dh1) @ A2 + np.abs(W["b2"]))
    dyv = forward_error_bound(p, X)
    r = y - np.asarray(target, dtype=np.float64)
    dy = (2.0 / B) * r
    ddy = (2.0 / B) * dyv + 2.0 ** -22 * np.abs(dy)
    Ady = np.abs(dy) + ddy
    # hidden backward signal d2 (rounded to BF16); masks uncertain where |z2| <= dz2
    d2 = dy[:, None] * w3[None, :] * (z2 > 0)
    flip2 = np.abs(z2) <= dz2
    Dd2 = np.where(flip2, (1.0 + u) * Ady[:, None] * np.abs(w3)[None, :],
                   (1.0 + u) * ddy[:, None] * np.abs(w3)[None, :] + u * np.abs(d2))
    Ad2 = np.abs(d2) + Dd2
    acc_t = 2.0 ** -15 + nb * 2.0 ** -24           # a tile's tensor-core sum, then the tile sum
    acc_c = (tile + nb) * 2.0 ** -24                # FP32 sums over a tile, then the tile sum
    Ah1 = np.abs(h1) + Dh1
    b = {}
    b["W2"] = Dh1.T @ Ad2 + np.abs(h1).T @ Dd2 + acc_t * (Ah1.T @ Ad2)
    b["b2"] = Dd2.sum(axis=0) + acc_t * Ad2.sum(axis=0)
    Ah2 = np.abs(h2) + dz2
    b["W3"] = (dz2.T @ Ady + np.abs(h2).T @ ddy + acc_c * (Ah2.T @ Ady))[:, None]
    b["b3"] = np.array([ddy.sum() + acc_c * Ady.sum()])
    # first-layer backward signal d1 = (d2 W2^T) [z1 > 0]
    d1pre = d2 @ W["W2"].T
    Dd1pre = Dd2 @ A2.T + 2.0 ** -16 * (Ad2 @ A2.T)
    flip1 = np.abs(z1) <= e1
    d1 = d1pre * (z1 > 0)
    Dd1 = np.where(flip1, np.abs(d1pre) + Dd1pre, Dd1pre)
    Ad1 = np.abs(d1) + Dd1
    b["W1"] = np.abs(X).T @ Dd1 + acc_c * (np.abs(X).T @ Ad1)
    b["b1"] = Dd1.sum(axis=0) + acc_c * Ad1.sum(axis=0)
    bl = float(np.mean(2.0 * np.abs(r) * dyv + dyv * dyv) + acc_c * np.mean((np.abs(r) + dyv) ** 2))
    return {k: v + 1e-30 for k, v in b.items()}, bl + 1e-30


def _bf16_ulp(a):
    """Spacing of BF16 numbers at |a| (2^(floor(log2 |a|) - 7)); 0 where a == 0."""
    a = np.abs(a)
    nz = a > 0
    return np.where(nz, np.exp2(np.floor(np.log2(np.where(nz, a, 1.0))) - 7), 0.0)


def gradient_rounding_sigma(p, X, target):
    """Standard deviation of each gradient entry's change when every first-layer
    activation h1 and every hidden backward signal d2 = dy W3^T [z2 > 0] is rounded to
    the nearest BF16 value, the errors taken as independent and uniform over half an
    ulp (variance ulp^2 / 12), to first order; a hidden ReLU mask near zero flips with
    the probability that the summed h1 roundings (normal approximation) cross it.  The
    h1 errors reach the gradient directly and through y (so through dy = 2 (y - t) / B,
    with dy/dh1_j = g_j = sum_k W2_jk [z2_k > 0] W3_k) and through z2 (so through h2)."""
    y, (X, z1, h1, z2, h2, W) = forward(p, X, round_weights=True)
    B = X.shape[0]
    w3 = W["W3"][:, 0]
    W2 = W["W2"]
    m2 = (z2 > 0).astype(np.float64)
    m1 = (z1 > 0).astype(np.float64)
    dy = (2.0 / B) * (y - np.asarray(target, dtype=np.float64))
    d2 = dy[:, None] * w3[None, :] * m2
    vh = _bf16_ulp(h1) ** 2 / 12.0                      # var of the h1 roundings [B, 64]
    # a z2 mask flips with probability Phi(-|z2| / sd(z2 change)) (normal approximation of
    # the summed h1 roundings), moving d2 by its whole value dy W3: variance p (dy W3)^2
    sz2 = np.sqrt(vh @ (W2 * W2))
    pf = 0.5 * erfc(np.abs(z2) / np.maximum(sz2, 1e-300) / np.sqrt(2.0))
    vd = _bf16_ulp(d2) ** 2 / 12.0 + pf * (dy[:, None] * w3[None, :]) ** 2   # d2 roundings and flips
    g = (W2[None, :, :] * (m2 * w3[None, :])[:, None, :]).sum(-1)   # dy/dh1 [B, 64]
    vdy = (2.0 / B) ** 2 * (vh * g * g).sum(1)           # var of the dy change [B]
    c = (2.0 / B) * m2 * w3[None, :]                     # d(d2_k)/d(y)  [B, 64]
    s2 = {}
    # dW2_jk = sum_s h1_sj d2_sk: the h1_sj rounding directly and via y; the d2 rounding
    Gd = np.einsum("sj,sk->jk", vh, d2 * d2)
    Gx = 2.0 * np.einsum("sj,sk->jk", vh * g * h1, d2 * c)
    Gy = np.einsum("sj,sk->jk", h1 * h1, (c * c) * (vh * g * g).sum(1)[:, None])
    Gr = np.einsum("sj,sk->jk", h1 * h1, vd)
    s2["W2"] = Gd + Gx + Gy + Gr
    s2["b2"] = ((c * c) * (vh * g * g).sum(1)[:, None] + vd).sum(0)
    # dW3_k = sum_s h2_sk dy_s: h2 moves through z2 (sum_j dh1_j W2_jk), dy through y
    a = dy[:, None, None] * m2[:, None, :] * W2[None, :, :] + h2[:, None, :] * (2.0 / B) * g[:, :, None]
    s2["W3"] = np.einsum("sj,sjk->k", vh, a * a)[:, None]
    s2["b3"] = np.array([vdy.sum()])
    # d1_sj = [z1_sj > 0] sum_k W2_jk d2_sk: the d2 changes through dy and their roundings
    q = (W2[None, :, :] * (m2 * w3[None, :])[:, None, :]).sum(-1)   # sum_k W2_jk m_k w3_k [B, 64]
    vd1 = m1 * ((2.0 / B) ** 2 * q * q * (vh * g * g).sum(1)[:, None] + vd @ (W2 * W2).T)
    s2["W1"] = (X * X).T @ vd1
    s2["b1"] = vd1.sum(0)
    return {k: np.sqrt(v) + 1e-30 for k, v in s2.items()}


def cv_coefficients(csr, T, t, xhat):
    """c3 = (xhat - T2)/t^3, a = A^3 v/2 - 3 c3, b = A c3."""
    T2 = T[0] + t * T[1] + t * t * T[2] / 2.0
    c3 = (np.asarray(xhat, dtype=np.float64) - T2) / t ** 3
    a = T[3] / 2.0 - 3.0 * c3
    b = _sp(csr) @ c3
    return c3, a, b
