"""Deterministic FP64 references for x = exp(tA) v (test infrastructure only).

Every function here is a direct, unblocked statement of a textbook definition;
library calls are limited to dense/sparse matrix products and the discrete
sine transform written out as a dense matrix.

Parity pins for these functions live in tests/test_oracle_dense.py:
closed forms (diagonal A, 2x2 symmetric, 2-state CTMC, cycle graph, complete
graph), mutual agreement of four independent methods, row-sum conservation of
CTMC generators, and SciPy's expm as an outside check.
"""
from __future__ import annotations

import math

import numpy as np


# ---------------------------------------------------------------------------
# O1: dense expm by scaling and squaring of a Taylor polynomial
# (Moler & Van Loan, "Nineteen dubious ways to compute the exponential of a
# matrix", method 3).  The problem statement of Sec. 2 is x = e^{beta A} v.
# ---------------------------------------------------------------------------

def expm_dense(a: np.ndarray) -> np.ndarray:
    """exp(a) for a dense square matrix, FP64.

    Scale by 2^-s so that the 1-norm is at most 1/2, sum the Taylor series
    until a term no longer changes the sum in FP64, then square s times.
    """
    a = np.asarray(a, dtype=np.float64)
    n = a.shape[0]
    norm = np.abs(a).sum(axis=0).max() if n else 0.0
    s = 0
    if norm > 0.5:
        s = int(math.ceil(math.log2(norm / 0.5)))
    b = a / (2.0 ** s)
    out = np.eye(n)
    term = np.eye(n)
    for k in range(1, 200):
        term = term @ b / k
        out = out + term
        if np.abs(term).max() <= 2.0 ** -60 * np.abs(out).max():
            break
    for _ in range(s):
        out = out @ out
    return out


def expmv_dense(a: np.ndarray, t: float, v: np.ndarray) -> np.ndarray:
    return expm_dense(t * np.asarray(a, dtype=np.float64)) @ np.asarray(v, dtype=np.float64)


# ---------------------------------------------------------------------------
# O2: Kronecker / discrete-sine closed form for Dirichlet grid Laplacians.
# Delta_h = T (+) T (+) T with T = h^-2 tridiag(1, -2, 1) of size m, whose
# eigenvectors are S_jk = sqrt(2/(m+1)) sin(j k pi/(m+1)) and eigenvalues
# mu_k = -4 h^-2 sin^2(k pi / (2(m+1))).  Hence exp(t Delta_h) = E (x) E (x) E
# with E = S diag(e^{t mu}) S.
# ---------------------------------------------------------------------------

def _grid_factor(m: int, t: float) -> np.ndarray:
    h = 1.0 / (m + 1)
    j = np.arange(1, m + 1)
    s = math.sqrt(2.0 / (m + 1)) * np.sin(np.outer(j, j) * math.pi / (m + 1))
    mu = -4.0 / (h * h) * np.sin(j * math.pi / (2.0 * (m + 1))) ** 2
    return s @ np.diag(np.exp(t * mu)) @ s


def grid2d_expmv(m: int, t: float, v: np.ndarray) -> np.ndarray:
    """exp(t Delta_h) v for the 5-point Dirichlet Laplacian; v indexed iy*m+ix."""
    e = _grid_factor(m, t)
    x = np.asarray(v, dtype=np.float64).reshape(m, m)  # [iy, ix]
    return (e @ x @ e.T).ravel()


def grid3d_expmv(m: int, t: float, v: np.ndarray, rows: np.ndarray | None = None) -> np.ndarray:
    """exp(t Delta_h) v for the 7-point Dirichlet Laplacian; v indexed (iz*m+iy)*m+ix.

    With ``rows`` given, only those entries are returned (each is one
    contraction of the rank-1-per-axis factor with v).
    """
    e = _grid_factor(m, t)
    x = np.asarray(v, dtype=np.float64).reshape(m, m, m)  # [iz, iy, ix]
    if rows is None:
        y = np.einsum("ai,ijk->ajk", e, x)
        y = np.einsum("bj,ajk->abk", e, y)
        y = np.einsum("ck,abk->abc", e, y)
        return y.ravel()
    rows = np.asarray(rows, dtype=np.int64)
    iz, rem = np.divmod(rows, m * m)
    iy, ix = np.divmod(rem, m)
    out = np.empty(rows.size)
    for q in range(rows.size):
        w = np.tensordot(e[iz[q]], x, axes=(0, 0))  # [iy, ix]
        w = e[iy[q]] @ w  # [ix]
        out[q] = e[ix[q]] @ w
    return out


# ---------------------------------------------------------------------------
# O3: truncated Taylor with scaling for large sparse A (the series of e^{tA}
# applied to v in s sub-steps, each stopped once a term is below 2^-53 of the
# partial sum in the infinity norm).
# ---------------------------------------------------------------------------

def taylor_expmv(a, t: float, v: np.ndarray, norm_bound: float | None = None) -> np.ndarray:
    """exp(tA) v for a scipy.sparse (or dense) A by s Taylor sub-steps of size t/s.

    s is chosen so that t * ||A||_1 / s <= 1.
    """
    v = np.asarray(v, dtype=np.float64)
    if norm_bound is None:
        norm_bound = float(abs(a).sum(axis=0).max()) if a.shape[0] else 0.0
    s = max(1, int(math.ceil(abs(t) * norm_bound)))
    h = t / s
    x = v.copy()
    for _ in range(s):
        term = x.copy()
        acc = x.copy()
        for k in range(1, 400):
            term = (a @ term) * (h / k)
            acc = acc + term
            if np.abs(term).max() <= 2.0 ** -53 * np.abs(acc).max():
                break
        x = acc
    return x


# ---------------------------------------------------------------------------
# O4: uniformization for CTMC generators Q (rows sum to 0, off-diagonal >= 0):
# exp(tQ) v = sum_k Pois(Lambda t; k) P^k v with P = I + Q/Lambda and
# Lambda >= max_i |q_ii|.  All terms are non-negative for v >= 0.
# ---------------------------------------------------------------------------

def uniformization_expmv(q, t: float, v: np.ndarray, tail: float = 1e-16) -> np.ndarray:
    import scipy.sparse as sp

    q = sp.csr_matrix(q)
    lam = float(np.max(-q.diagonal())) if q.shape[0] else 0.0
    if lam <= 0.0 or t == 0.0:
        return np.asarray(v, dtype=np.float64).copy()
    p = sp.identity(q.shape[0], format="csr") + q / lam
    mu = lam * t
    # Poisson weights computed in log space, summed until the remaining tail mass is below `tail`
    term = np.asarray(v, dtype=np.float64).copy()
    out = np.zeros_like(term)
    k = 0
    cum = 0.0
    kmax = int(mu + 40.0 * math.sqrt(mu + 1.0) + 100)
    while k <= kmax:
        w = math.exp(-mu + k * math.log(mu) - math.lgamma(k + 1)) if mu > 0 else (1.0 if k == 0 else 0.0)
        out += w * term
        cum += w
        if k > mu and 1.0 - cum < tail:
            break
        term = p @ term
        k += 1
    return out


# ---------------------------------------------------------------------------
# O5: the split targets of Sec. 2.  With A = D - L, D = diag(delta) and
#   Lie    (Eq. deff):        x^L = (e^{-dt L} e^{dt D})^N v,
#   Strang (Eq. eq_general1): x^S = (e^{dt D/2} e^{-dt L} e^{dt D/2})^N v,
# where dt = t/N.  delta_i is the full row sum of A (the potential) and -L is
# the generator with off-diagonals a_ij and diagonal -sum_{j!=i} a_ij.
# ---------------------------------------------------------------------------

def split_decompose(a: np.ndarray):
    """Return (delta, Qgen) with A = diag(delta) + Qgen and Qgen a generator."""
    a = np.asarray(a, dtype=np.float64)
    off = a - np.diag(np.diag(a))
    lam = off.sum(axis=1)
    delta = np.diag(a) + lam
    qgen = off - np.diag(lam)
    return delta, qgen


def split_expmv(a: np.ndarray, t: float, nsteps: int, v: np.ndarray, kind: str) -> np.ndarray:
    delta, qgen = split_decompose(a)
    dt = t / nsteps
    p = expm_dense(dt * qgen)  # e^{-dt L}
    x = np.asarray(v, dtype=np.float64).copy()
    if kind == "lie":
        ed = np.exp(dt * delta)
        for _ in range(nsteps):
            x = p @ (ed * x)
    elif kind == "strang":
        eh = np.exp(0.5 * dt * delta)
        for _ in range(nsteps):
            x = eh * (p @ (eh * x))
    else:
        raise ValueError(kind)
    return x


# ---------------------------------------------------------------------------
# a10: power iteration for lambda_max (Sec. 6 uses beta = 1/lambda_max).
# ---------------------------------------------------------------------------

def power_iteration(a, iters: int = 1000, tol: float = 1e-12, x0: np.ndarray | None = None) -> float:
    """Largest eigenvalue of a symmetric non-negative matrix by the power method.

    Starts from the all-ones vector; returns the Rayleigh quotient once two
    successive estimates agree to ``tol`` relative.
    """
    n = a.shape[0]
    x = np.ones(n) if x0 is None else np.asarray(x0, dtype=np.float64).copy()
    x /= np.linalg.norm(x)
    lam = 0.0
    for _ in range(iters):
        y = a @ x
        new = float(x @ y)
        ny = np.linalg.norm(y)
        if ny == 0.0:
            return 0.0
        x = y / ny
        if abs(new - lam) <= tol * abs(new):
            return new
        lam = new
    return lam
