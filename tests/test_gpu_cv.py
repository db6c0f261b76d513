"""GPU parity of the learned control variate (Sec. 5: variance reduction).

* Taylor terms and node features against oracle/cv.py.
* The network on the tensor cores: predictions and full-batch gradients against
  the plain FP64 forward pass and gradient with the same BF16-rounded weights,
  within the derived bounds and with the mean square difference one
  round-to-nearest spread; Adam training that drives the loss down.
* The CV walker on the same paths as the oracle's CV estimator: FP64 residual
  integrals within 1e-12, FP32 within 1e-5 of the entry's scale.
* Unbiasedness for an arbitrary prediction (z-test against expm), zero
  variance when h is exact, and the gain of the trained network over plain
  MC and over the Taylor-only control variate at equal paths.
"""
import math

import numpy as np
import pytest

import workloads as W
import zstats
from oracle import cv as CV
from oracle import dense as OD
from oracle import walker as OW

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def mcx():
    import paper_1904_12759_gb300 as P

    P.load()
    return P


def _dev(csr):
    return (torch.as_tensor(csr.row_ptr).cuda(), torch.as_tensor(csr.col).cuda(), torch.as_tensor(csr.val).cuda())


def _conditioned(n, seed, rate=1.5, dsd=1.0):
    rng = np.random.default_rng(seed)
    a = np.where(rng.random((n, n)) < 0.3, rng.lognormal(0, 1, (n, n)), 0.0)
    np.fill_diagonal(a, 0.0)
    a *= rate / a.sum(axis=1).mean()
    np.fill_diagonal(a, rng.normal(0, dsd, n) - a.sum(axis=1) + rng.normal(0, dsd, n))
    return a


def _fp64_bound(csr, v):
    """Error bound of the Taylor terms A^k v on either side (FP64 row sums in
    different orders: each of the k chained row sums is exact to
    (row length + 1) 2^-53 of its absolute sum, so |T_k - A^k v| <=
    2 * 3 (maxdeg + 1) 2^-52 (|A|^k |v|) between the two), as [4, n]."""
    a = abs(csr.to_scipy())
    S = [np.abs(np.asarray(v, dtype=np.float64))]
    for _ in range(3):
        S.append(a @ S[-1])
    return 6 * (np.diff(csr.row_ptr).max() + 1) * 2.0 ** -52 * np.stack(S)


def _with_hub(csr):
    """The graph plus one node joined to every other node (a row of n - 1 entries)."""
    import scipy.sparse as sp

    n = csr.n
    a = csr.to_scipy().tolil()
    a.resize((n + 1, n + 1))
    a[n, :n] = 1.0
    a[:n, n] = 1.0
    m = sp.csr_matrix(a)
    m.sort_indices()
    return W.CSR(n + 1, m.indptr.astype(np.int64), m.indices.astype(np.int32), m.data.astype(np.float64))


def _mixed_rows(n=2037, seed=6, signed=True):
    """A CSR with every row class of the row passes and a ragged last window: empty
    rows, short rows, rows of 33..1024 entries and one above 1024 (a hub); values of
    both signs (negative off-diagonal entries do not count in the rates), or with
    signed=False nonnegative off the diagonal (a matrix the walkers accept)."""
    import scipy.sparse as sp

    rng = np.random.default_rng(seed)
    a = sp.random(n, n, density=4.0 / n, random_state=seed, format="lil")
    a[5, rng.choice(n, min(1500, n - 1), replace=False)] = 1.0
    for i in (17, 400, n - 40):
        a[i, rng.choice(n, 40 + i % 300, replace=False)] = 0.5
    a = sp.csr_matrix(a)
    a.data = rng.normal(size=a.data.size)
    if not signed:
        r, c = a.nonzero()
        a.data = np.where(r == c, a.data, np.abs(a.data))
    a = a.tolil()
    for i in range(0, n, 9):  # every 9th row empty
        a.rows[i] = []
        a.data[i] = []
    m = sp.csr_matrix(a)
    m.sort_indices()
    return W.CSR(n, m.indptr.astype(np.int64), m.indices.astype(np.int32), m.data.astype(np.float64))


def test_prepare_and_coefficients_on_every_row_class(mcx):
    """Taylor terms, features and coefficients on a matrix with empty, short, long and
    hub rows and a ragged last window of the row schedule, against the oracle."""
    csr = _mixed_rows()
    deg = np.diff(csr.row_ptr)
    assert deg.min() == 0 and deg.max() > 1024 and np.any((deg > 32) & (deg <= 1024)) and csr.n % 256
    v = W.uniform_vector(csr.n, 3, -1.0, 1.0)
    t = 0.05
    rp, col, val = _dev(csr)
    T, F = mcx.cv_prepare(rp, col, val, torch.as_tensor(v).cuda(), t)
    oF, _, oT = CV.features(csr, v, t)
    assert np.all(np.abs(T.cpu().numpy() - oT) <= _fp64_bound(csr, v))
    assert np.allclose(F.cpu().numpy(), oF.astype(np.float32), rtol=2e-6, atol=1e-6)
    y = torch.as_tensor(np.random.default_rng(2).normal(0, 0.3, csr.n).astype(np.float32)).cuda()
    coef = mcx.cv_coefficients(rp, col, val, T, y, t).cpu().numpy()
    T2 = oT[0] + t * oT[1] + t * t * oT[2] / 2
    xhat = T2 * np.exp(y.cpu().numpy().astype(np.float64))
    _, ca, cb = CV.cv_coefficients(csr, oT, t, xhat)
    B = _fp64_bound(csr, v)
    assert np.all(np.abs(coef[2 * csr.n:] - xhat) <= 1e-15 * np.abs(xhat) + np.exp(y.cpu().numpy()) *
                  (t * B[1] + t * t * B[2] / 2) + 1e-300)
    ab = coef[:2 * csr.n].reshape(csr.n, 2)
    assert np.allclose(ab[:, 0], ca, rtol=1e-11, atol=1e-12 * np.abs(ca).max())
    assert np.allclose(ab[:, 1], cb, rtol=1e-10, atol=1e-11 * np.abs(cb).max())


@pytest.mark.parametrize("scale", [1.0, 3e-26])  # 3e-26: rates below 2^-74, the FP64 feature sums
def test_prepare_matches_oracle(mcx, scale):
    import dataclasses

    # rows of 33..1024 entries take the warp-per-row kernels, the added hub (2999) the block-per-row ones
    csr = _with_hub(W.barabasi_albert(2999, 5, 4))
    deg = np.diff(csr.row_ptr)
    assert deg.max() > 1024 and np.any((deg > 32) & (deg <= 1024))
    csr = dataclasses.replace(csr, val=csr.val * scale)
    v = W.uniform_vector(3000, 1)
    t = 0.03
    rp, col, val = _dev(csr)
    T, F = mcx.cv_prepare(rp, col, val, torch.as_tensor(v).cuda(), t)
    oF, oT2, oT = CV.features(csr, v, t)
    assert np.all(np.abs(T.cpu().numpy() - oT) <= _fp64_bound(csr, v))
    assert np.array_equal(T.cpu().numpy()[0], v)
    assert np.allclose(F.cpu().numpy(), oF.astype(np.float32), rtol=2e-6, atol=1e-6 * scale)


def test_coefficient_exponential_within_two_ulp(mcx):
    """xhat = T2 e^y with T2 = 1 (v = 1, Av = A^2 v = 0): the coefficients' FP64
    exponential of the network's FP32 output against numpy's, within 2 units in
    the last place, over [-30, 30], the reduction's edges (multiples of ln(2)/64
    and halfway between), and the range ends (|y| >= 700 takes the library's
    exponential; overflow to inf, underflow to 0)."""
    rng = np.random.default_rng(4)
    k = np.arange(-40, 41)
    edges = np.concatenate([k * math.log(2) / 64, (k + 0.5) * math.log(2) / 64])
    special = [0.0, 1e-30, -1e-30, 2.0 ** -20, -(2.0 ** -20), 88.0, -88.0, 699.9, -699.9, 700.0, -700.0, 705.0,
               -705.0, 709.7, 710.0, -708.0, -760.0, 1000.0]
    y = np.concatenate([rng.uniform(-30, 30, 200000), edges, special]).astype(np.float32)
    n = y.size
    taylor = torch.zeros(4 * n, dtype=torch.float64, device="cuda")
    taylor[:n] = 1.0
    rp = torch.arange(n + 1, dtype=torch.int64, device="cuda")
    col = torch.arange(n, dtype=torch.int32, device="cuda")
    val = torch.ones(n, dtype=torch.float64, device="cuda")
    coef = mcx.cv_coefficients(rp, col, val, taylor, torch.as_tensor(y).cuda(), 0.5)
    h = coef[2 * n:].cpu().numpy()
    with np.errstate(over="ignore"):
        e = np.exp(y.astype(np.float64))
    fin = np.isfinite(e) & (e > 0)
    assert np.all(np.abs(h[fin] - e[fin]) <= 2 * np.spacing(e[fin])), \
        np.max(np.abs(h[fin] - e[fin]) / np.spacing(e[fin]))
    assert np.all(h[~fin] == e[~fin])


def test_network_forward_and_gradient_match_oracle(mcx):
    rng = np.random.default_rng(2)
    X = rng.normal(size=(777, 5)).astype(np.float32)  # ragged: not a multiple of 64
    tgt = rng.normal(size=777).astype(np.float32)
    net = mcx.MLP(seed=5)
    p = CV.init_params(9)
    flat = np.concatenate([p["W1"].ravel(), p["b1"], p["W2"].ravel(), p["b2"], p["W3"].ravel(), p["b3"]])
    net.set(flat, np.zeros(5), np.ones(5))
    y = net.predict(torch.as_tensor(X).cuda()).cpu().numpy()
    net.sync()
    # tensor-core inference against the plain FP64 forward pass (same BF16 weights): every
    # node within the derived bound of one BF16 rounding per first-layer activation plus
    # FP32 accumulation, and the mean square difference in units of the round-to-nearest
    # spread near 1 (rounding toward zero, a wrong rounding rule, gives more than 2)
    X64 = X.astype(np.float64)
    oy, _ = CV.forward(p, X64, round_weights=True)
    d = y.astype(np.float64) - oy
    assert np.all(np.abs(d) <= CV.forward_error_bound(p, X64)), np.max(np.abs(d) / CV.forward_error_bound(p, X64))
    ms = float(np.mean((d / CV.forward_rounding_sigma(p, X64)) ** 2))
    assert 0.6 < ms < 1.6, ms
    # gradient on the tensor cores (h1 and the hidden backward signal in BF16, FP32
    # accumulation) against the FP64 gradient with the same BF16 weights: every entry
    # within the derived bound, and the mean square of the differences in units of the
    # round-to-nearest spread of those two roundings near 1 (truncation gives > 10)
    g, loss = net.gradient(torch.as_tensor(X).cuda(), torch.as_tensor(tgt).cuda())
    g = g.cpu().numpy()
    T64 = tgt.astype(np.float64)
    oloss, og = CV.loss_and_grad(p, X64, T64, round_weights=True)
    gb, lb = CV.gradient_error_bound(p, X64, T64)
    sig = CV.gradient_rounding_sigma(p, X64, T64)
    assert abs(loss - oloss) <= lb
    order = ("W1", "b1", "W2", "b2", "W3", "b3")
    ogf = np.concatenate([og[k].ravel() for k in order])
    bf = np.concatenate([gb[k].ravel() for k in order])
    sf = np.concatenate([sig[k].ravel() for k in order])
    assert np.all(np.abs(g - ogf) <= bf), np.max(np.abs(g - ogf) / bf)
    ms = float(np.mean(((g - ogf) / sf) ** 2))
    assert 0.4 < ms < 3.0, ms
    net.close()


def test_training_reduces_loss(mcx):
    rng = np.random.default_rng(0)
    X = rng.normal(size=(20000, 5)).astype(np.float32)
    tgt = (np.sin(X[:, 0]) + 0.5 * X[:, 1] * X[:, 2] - 0.3 * X[:, 3] ** 2).astype(np.float32)
    net = mcx.MLP(seed=1)
    losses = net.fit(torch.as_tensor(X).cuda(), torch.as_tensor(tgt).cuda(), epochs=15, batch=1024, lr=3e-3, seed=2)
    assert losses[-1] < 0.2 * losses[0], losses
    net.close()


@pytest.mark.parametrize("M", [3000, 40])  # warp-per-entry and lane-per-entry layouts
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_cv_estimates_match_oracle_same_paths(mcx, prec, M):
    a = _conditioned(80, 21)
    csr = W.dense_to_csr(a)
    v = W.uniform_vector(80, 2, -1.0, 1.0)
    t = 0.8
    rp, col, val = _dev(csr)
    T, F = mcx.cv_prepare(rp, col, val, torch.as_tensor(v).cuda(), t)
    yrand = torch.as_tensor(np.random.default_rng(3).normal(0, 0.5, 80).astype(np.float32)).cuda()
    coef = mcx.cv_coefficients(rp, col, val, T, yrand, t)
    # oracle coefficients from the same prediction
    oT = CV.taylor_terms(csr, v)
    T2 = oT[0] + t * oT[1] + t * t * oT[2] / 2
    xhat = T2 * np.exp(yrand.cpu().numpy().astype(np.float64))
    c3, ca, cb = CV.cv_coefficients(csr, oT, t, xhat)
    cg = coef.cpu().numpy()
    # xhat = T2 e^y inherits the Taylor terms' bound
    B = _fp64_bound(csr, v)
    ey = np.exp(yrand.cpu().numpy().astype(np.float64))
    assert np.all(np.abs(cg[160:] - xhat) <= 1e-15 * np.abs(xhat) + ey * (t * B[1] + t * t * B[2] / 2))
    assert np.allclose(cg[:160].reshape(80, 2), np.stack([ca, cb], 1), rtol=1e-11, atol=1e-12 * np.abs(ca).max())
    plan = mcx.Plan.from_csr(csr)
    gm, gs = plan.estimate_cv(coef, t, M, seed=7, prec=prec)
    # the walker is compared on the GPU's own coefficients (checked above)
    gab = cg[:160].reshape(80, 2)
    om, os_ = OW.Graph(csr).estimate_cv(gab[:, 0].copy(), gab[:, 1].copy(), cg[160:].copy(), t, M, seed=7)
    gm, gs = gm.cpu().numpy(), gs.cpu().numpy()
    scale = np.abs(xhat) + os_ * math.sqrt(M)
    tol = 1e-12 if prec == "fp64" else 1e-5
    assert np.all(np.abs(gm - om) <= tol * scale), np.max(np.abs(gm - om) / scale)
    assert np.allclose(gs, os_, rtol=1e-9 if prec == "fp64" else 1e-3)
    if M >= 1000:  # unbiased for this arbitrary prediction
        zstats.check((gm - OD.expmv_dense(a, t, v)) / gs, samples=M)
    plan.close()


@pytest.mark.parametrize("M", [3000, 40])  # warp-per-entry and lane-per-entry layouts
@pytest.mark.parametrize("vscale", [1e-30, 1e30])
def test_cv_fp32_integrals_at_any_scale_of_v(mcx, M, vscale):
    """FP32 residual integrals read the coefficients scaled by a power of two (exact), so
    v scaled by 1e-30 or 1e30 gives estimates and standard errors that match the oracle
    as v itself does: no squared residual underflows to a zero standard error, none
    overflows.  The scale of the comparison adds the estimate of the absolute
    integrand (|a|, |b|) on the same paths, what the FP32 sums add up."""
    a = _conditioned(80, 21)
    csr = W.dense_to_csr(a)
    v = W.uniform_vector(80, 2, -1.0, 1.0) * vscale
    t = 0.8
    rp, col, val = _dev(csr)
    T, F = mcx.cv_prepare(rp, col, val, torch.as_tensor(v).cuda(), t)
    yrand = torch.as_tensor(np.random.default_rng(3).normal(0, 0.5, 80).astype(np.float32)).cuda()
    coef = mcx.cv_coefficients(rp, col, val, T, yrand, t)
    plan = mcx.Plan.from_csr(csr)
    gm, gs = plan.estimate_cv(coef, t, M, seed=7, prec="fp32")
    cg = coef.cpu().numpy()
    ab = cg[:160].reshape(80, 2)
    og = OW.Graph(csr)
    om, os_ = og.estimate_cv(ab[:, 0].copy(), ab[:, 1].copy(), cg[160:].copy(), t, M, seed=7)
    habs, _ = og.estimate_cv(np.abs(ab[:, 0]), np.abs(ab[:, 1]), np.zeros(80), t, M, seed=7)
    gm, gs = gm.cpu().numpy(), gs.cpu().numpy()
    scale = np.abs(cg[160:]) + os_ * math.sqrt(M) + habs
    assert np.all(np.abs(gm - om) <= 1e-5 * scale), np.max(np.abs(gm - om) / scale)
    assert np.allclose(gs, os_, rtol=1e-3, atol=1e-6 * scale.max()) and np.all(gs[os_ > 0] > 0)
    assert plan.sync()["status_bits"] == 0
    plan.close()


def test_cv_exact_h_zero_variance(mcx):
    a = np.zeros((3, 3))
    a[0, 1] = 1.3
    a[1, 2] = 0.7
    csr = W.dense_to_csr(a)
    v = np.array([0.2, 1.0, 2.0])
    rp, col, val = _dev(csr)
    T, _ = mcx.cv_prepare(rp, col, val, torch.as_tensor(v).cuda(), 0.9)
    coef = mcx.cv_coefficients(rp, col, val, T, None, 0.9)
    plan = mcx.Plan.from_csr(csr)
    m, s = plan.estimate_cv(coef, 0.9, 4096, prec="fp64")
    assert np.allclose(m.cpu().numpy(), OD.expmv_dense(a, 0.9, v), rtol=1e-13)
    assert torch.all(s == 0)
    plan.close()


def test_learned_cv_gain_over_plain_and_taylor(mcx):
    """Train on labels from the Taylor-only control-variate estimator on two small BA
    graphs (the method's own estimates), then on a third graph compare, at equal
    paths, the relative L2 error of plain MC, the Taylor-only CV and the learned CV
    against the FP64 Taylor oracle; unbiasedness is checked with many paths on a
    subset (per-path weights are skewed, so z-scores need large samples)."""
    def setup(seed, n=20000):
        csr = W.barabasi_albert(n, 5, seed)
        v = W.uniform_vector(n, seed + 100)
        lam = OD.power_iteration(csr.to_scipy(), iters=2000, tol=1e-10)
        return csr, v, 0.5 / lam

    feats, tgts = [], []
    for seed in (1, 2):
        csr, v, t = setup(seed)
        rp, col, val = _dev(csr)
        vd = torch.as_tensor(v).cuda()
        plan = mcx.Plan.from_csr(csr)
        T, F = mcx.cv_prepare(rp, col, val, vd, t)
        x, _ = plan.estimate_cv(mcx.cv_coefficients(rp, col, val, T, None, t), t, 256, seed=seed)
        feats.append(F)
        tgts.append(mcx.cv_targets(x, T, t))
        plan.close()
    net = mcx.MLP(seed=3)
    losses = net.fit(torch.cat(feats), torch.cat(tgts), epochs=30, batch=2048, lr=2e-3, seed=4)
    assert losses[-1] < 0.5 * losses[0]
    csr, v, t = setup(7)
    rp, col, val = _dev(csr)
    vd = torch.as_tensor(v).cuda()
    plan = mcx.Plan.from_csr(csr)
    T, F = mcx.cv_prepare(rp, col, val, vd, t)
    x = OD.taylor_expmv(csr.to_scipy(), t, v)
    M = 64
    m_pl, s_pl = plan.estimate(vd, t, M, seed=9)
    coef_tay = mcx.cv_coefficients(rp, col, val, T, None, t)
    coef_cv = mcx.cv_coefficients(rp, col, val, T, net.predict(F), t)
    m_tay, s_tay = plan.estimate_cv(coef_tay, t, M, seed=9)
    m_cv, s_cv = plan.estimate_cv(coef_cv, t, M, seed=9)
    err = lambda m: float(np.linalg.norm(m.cpu().numpy() - x) / np.linalg.norm(x))  # noqa: E731
    rms = lambda s: float(np.sqrt(np.mean(s.cpu().numpy() ** 2)))  # noqa: E731
    print(f"rel L2 error at M={M}: plain {err(m_pl):.3e} taylor-cv {err(m_tay):.3e} learned-cv {err(m_cv):.3e}; "
          f"rms SE plain {rms(s_pl):.3e} taylor {rms(s_tay):.3e} learned {rms(s_cv):.3e}")
    assert err(m_cv) < err(m_pl) / 10
    assert rms(s_cv) < rms(s_tay)  # the network helps beyond the Taylor-only control variate
    # unbiasedness with many paths on a subset
    ent = torch.as_tensor(W.random_entries(csr.n, 300, 5)).cuda()
    m, s = plan.estimate_cv(coef_cv, t, 20000, entries=ent, seed=11)
    zstats.check((m.cpu().numpy() - x[ent.cpu().numpy()]) / s.cpu().numpy(), samples=20000)
    plan.close()
    net.close()
