"""GPU parity of the batched control-variate form (mcx_cvbatch_*): many (A, v, t),
several right-hand sides per A, one graph launch per run.

* Every (problem, right-hand side) pair k simulates the paths k * 2^40 + p of the
  single-problem estimators, so its estimate is compared with the oracle's on the
  same paths: plain estimates (Theorem 1, Algorithm 1) within 2e-6 of the entry's
  scale (FP32 paths) or 1e-12 (FP64 paths); control-variate estimates within 1e-5
  (FP32 residual integrals) or 1e-12 (FP64) of |h| + SE sqrt(M), on the batch's own
  coefficients.
* The batch's pre-pass (Taylor terms, features, network, coefficients) equals the
  single-problem calls on the same inputs bit for bit.
* Uneven sizes, both layouts (lane per entry for M <= 64, warp per entry chunk
  above), weighted (alias-table) rows, several right-hand sides with different
  horizons and scales, several chunks per entry.
* Runs are deterministic given the seed; changing the paths re-lays the work out;
  the network is read at every run; the batched estimate is unbiased against
  expm (the three-part z rule of tests/zstats.py); invalid descriptions are rejected.
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


def _conditioned(n, seed, rate=1.5, dsd=1.0):
    rng = np.random.default_rng(seed)
    a = np.where(rng.random((n, n)) < 0.3, rng.lognormal(0, 1, (n, n)), 0.0)
    np.fill_diagonal(a, 0.0)
    a *= rate / a.sum(axis=1).mean()
    np.fill_diagonal(a, rng.normal(0, dsd, n) - a.sum(axis=1) + rng.normal(0, dsd, n))
    return a


def _problems():
    """Three problems of uneven sizes; 4 pairs.  Problem 0 (BA, 0/1 adjacency) has two
    right-hand sides of different horizons and scales and few paths (lane layout);
    problem 1 (weighted rows: alias tables) many paths per entry over a small n
    (several chunks per entry); problem 2 (ER) a single right-hand side, warp layout."""
    ba = W.barabasi_albert(1500, 3, 2)
    wt = W.dense_to_csr(_conditioned(120, 3))
    er = W.erdos_renyi(300, 6, 3)
    v0 = np.stack([W.uniform_vector(1500, 10), 1e-30 * W.uniform_vector(1500, 11, -1.0, 1.0)])
    return [
        dict(csr=ba, v=v0, t=np.array([0.05, 0.1]), paths=40),
        dict(csr=wt, v=W.uniform_vector(120, 12, -1.0, 1.0)[None], t=np.array([0.6]), paths=70000),
        dict(csr=er, v=W.uniform_vector(300, 13)[None], t=np.array([0.08]), paths=3000),
    ]


def _desc(probs):
    return [dict(row_ptr=p["csr"].row_ptr, col=p["csr"].col, val=p["csr"].val, v=p["v"], t=p["t"],
                 paths=p["paths"]) for p in probs]


def _net(mcx):
    net = mcx.MLP(seed=5)
    prm = CV.init_params(9)
    net.set(np.concatenate([prm[k].ravel() for k in ("W1", "b1", "W2", "b2", "W3", "b3")]), np.zeros(5), np.ones(5))
    return net


def _dev(csr):
    return (torch.as_tensor(csr.row_ptr).cuda(), torch.as_tensor(csr.col).cuda(), torch.as_tensor(csr.val).cuda())


@pytest.mark.parametrize("control", ["none", "taylor", "learned"])
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_cvbatch_pairs_match_oracle_on_the_same_paths(mcx, tmp_path, control, prec):
    probs = _problems()
    net = _net(mcx) if control == "learned" else None
    cache = str(tmp_path / "cvb.jsonl")
    b = mcx.CVBatch(_desc(probs), control=control, net=net, prec=prec, tune_cache=cache)
    info = b.info()
    assert info["pairs"] == 4 and info["problems"] == 3 and info["control"] == ["none", "taylor", "learned"].index(control)
    b.run(seed=7)
    k = 0
    for pb, p in enumerate(probs):
        csr, M = p["csr"], p["paths"]
        og = OW.Graph(csr)
        rp, col, val = _dev(csr)
        for r in range(p["v"].shape[0]):
            v, t = p["v"][r], float(p["t"][r])
            x, s = b.result(pb, r)
            x, s = x.cpu().numpy(), s.cpu().numpy()
            off = k << 40
            if control == "none":
                om, os_, _ = og.estimate(v, t, M, seed=7, path_offset=off, prec=prec)
                scale, _, _ = og.estimate(np.abs(v), t, M, seed=7, path_offset=off, prec=prec)
                tol = 1e-12 if prec == "fp64" else 2e-6
                assert np.all(np.abs(x - om) <= tol * scale), (pb, r, np.max(np.abs(x - om) / scale))
                # FP32: the variance comes from an FP32 sum of M squares minus the squared mean;
                # its rounding (~2^-23 of E[w^2]) leaves |dSE| <= scale sqrt(2^-22 / M) even
                # where the paths' spread is zero (an isolated node)
                assert np.allclose(s, os_, rtol=1e-9 if prec == "fp64" else 1e-3,
                                   atol=0 if prec == "fp64" else scale.max() * math.sqrt(2.0 ** -22 / M)), \
                    (pb, r, float(np.max(np.abs(s - os_) / np.maximum(np.abs(os_), 1e-300))), float(scale.max()))
            else:
                coef = b.coefficients(pb, r)
                # the pre-pass equals the single-problem calls on the same inputs, bit for bit
                T, F = mcx.cv_prepare(rp, col, val, torch.as_tensor(v).cuda(), t)
                y = net.predict(F) if control == "learned" else None
                assert torch.equal(coef, mcx.cv_coefficients(rp, col, val, T, y, t))
                cg = coef.cpu().numpy()
                n = csr.n
                ab = cg[:2 * n].reshape(n, 2)
                om, os_ = og.estimate_cv(ab[:, 0].copy(), ab[:, 1].copy(), cg[2 * n:].copy(), t, M, seed=7,
                                         path_offset=off)
                # scale: what the residual sums add up, |h| + SE sqrt(M) and the estimate of the
                # absolute integrand (|a|, |b|) on the same paths (FP32 integrals cancel in it)
                habs, _ = og.estimate_cv(np.abs(ab[:, 0]), np.abs(ab[:, 1]), np.zeros(n), t, M, seed=7,
                                         path_offset=off)
                scale = np.abs(cg[2 * n:]) + os_ * math.sqrt(M) + habs
                tol = 1e-12 if prec == "fp64" else 1e-5
                assert np.all(np.abs(x - om) <= tol * scale), (pb, r, np.max(np.abs(x - om) / scale))
                # the variance comes from sums of y and y^2 (FP32 squares for FP32 integrals):
                # rounding of the sum of squares leaves |dSE| <= scale sqrt(2^-22 / M) (FP32) or
                # scale sqrt(2^-50 / M) (FP64), also where the spread is zero
                assert np.allclose(s, os_, rtol=1e-6 if prec == "fp64" else 1e-3,
                                   atol=scale.max() * math.sqrt((2.0 ** -50 if prec == "fp64" else 2.0 ** -22) / M)), \
                    (pb, r, float(np.max(np.abs(s - os_) / np.maximum(np.abs(os_), 1e-300))), float(scale.max()))
                assert np.all(s[os_ > 0] > 0)  # no standard error lost to FP32 underflow
            k += 1
    st = b.sync()
    assert st["status_bits"] == 0
    assert st["paths"] == sum(p["paths"] * p["csr"].n * p["v"].shape[0] for p in probs)
    b.close()
    # the schedule was cached: a second batch of the same signature reads it back
    b2 = mcx.CVBatch(_desc(probs), control=control, net=net, prec=prec, tune_cache=cache)
    i2 = b2.info()
    assert i2["tuned_ms"] == 0.0 and (i2["chunk"], i2["blocks_per_sm"], i2["staged"]) == \
        (info["chunk"], info["blocks_per_sm"], info["staged"])
    b2.close()
    if net is not None:
        net.close()


def test_cvbatch_deterministic_paths_change_and_network_read_per_run(mcx):
    probs = _problems()
    net = _net(mcx)
    b = mcx.CVBatch(_desc(probs), control="learned", net=net)
    b.run(seed=3)
    x1 = [b.result(i, r)[0].clone() for i, p in enumerate(probs) for r in range(p["v"].shape[0])]
    b.run(seed=3)
    x2 = [b.result(i, r)[0].clone() for i, p in enumerate(probs) for r in range(p["v"].shape[0])]
    assert all(torch.equal(a, c) for a, c in zip(x1, x2))
    b.run(seed=4)
    assert not torch.equal(b.result(2)[0], x1[-1])
    # new paths per entry: problem 2 moves to the lane layout, problem 0 to the warp layout
    b.set_paths([200, 70000, 16])
    b.run(seed=3)
    og = OW.Graph(probs[2]["csr"])
    coef = b.coefficients(2).cpu().numpy()
    n = probs[2]["csr"].n
    ab = coef[:2 * n].reshape(n, 2)
    om, os_ = og.estimate_cv(ab[:, 0].copy(), ab[:, 1].copy(), coef[2 * n:].copy(), 0.08, 16, seed=3,
                             path_offset=3 << 40)
    x = b.result(2)[0].cpu().numpy()
    assert np.all(np.abs(x - om) <= 1e-5 * (np.abs(coef[2 * n:]) + os_ * 4))
    # the network's weights are read at every run
    before = b.result(0)[0].clone()
    prm, _, _ = net.get()
    prm[-1] += 0.25  # output bias: every prediction scales by e^0.25
    net.set(prm)
    b.run(seed=3)
    c0 = b.coefficients(0).cpu().numpy()
    assert not torch.equal(b.result(0)[0], before)
    assert b.sync()["status_bits"] == 0
    b.close()
    net.close()
    assert np.all(np.isfinite(c0))


def test_cvbatch_unbiased_against_expm(mcx):
    """Two weighted problems with arbitrary (untrained) predictions: the batched learned
    control-variate estimates have per-entry z-scores against expm with tail fraction,
    mean and variance within the bounds of tests/zstats.py."""
    a1, a2 = _conditioned(60, 31), _conditioned(90, 32)
    v1, v2 = W.uniform_vector(60, 1, 0.2, 1.0), W.uniform_vector(90, 2, -1.0, 1.0)
    probs = [dict(csr=W.dense_to_csr(a1), v=v1[None], t=np.array([0.7]), paths=20000),
             dict(csr=W.dense_to_csr(a2), v=v2[None], t=np.array([0.4]), paths=20000)]
    net = _net(mcx)
    b = mcx.CVBatch(_desc(probs), control="learned", net=net)
    b.run(seed=11)
    z = []
    for i, (a, v, t) in enumerate(((a1, v1, 0.7), (a2, v2, 0.4))):
        x, s = b.result(i)
        z.append((x.cpu().numpy() - OD.expmv_dense(a, t, v)) / s.cpu().numpy())
    zstats.check(np.concatenate(z), samples=20000)
    b.close()
    net.close()


def test_cvbatch_coefficients_bit_identical_on_every_row_class(mcx):
    """The batch's pre-pass (slot CSR, sliced ELL short rows, fused A^3 v / A c3 pass)
    gives the bits of the single-problem calls on matrices with empty, short, long and
    hub rows, for two problems with two right-hand sides each."""
    from test_gpu_cv import _mixed_rows

    csrs = [_mixed_rows(2037, 6, signed=False), _mixed_rows(1100, 7, signed=False)]
    probs = [dict(row_ptr=c.row_ptr, col=c.col, val=c.val,
                  v=np.stack([W.uniform_vector(c.n, 20 + i, -1.0, 1.0), W.uniform_vector(c.n, 30 + i)]),
                  t=np.array([0.05, 0.02]), paths=8) for i, c in enumerate(csrs)]
    net = _net(mcx)
    b = mcx.CVBatch(probs, control="learned", net=net)
    b.run(seed=1)
    for pb, c in enumerate(csrs):
        rp, col, val = _dev(c)
        for r in range(2):
            v, t = probs[pb]["v"][r], float(probs[pb]["t"][r])
            T, F = mcx.cv_prepare(rp, col, val, torch.as_tensor(v).cuda(), t)
            assert torch.equal(b.coefficients(pb, r), mcx.cv_coefficients(rp, col, val, T, net.predict(F), t))
    assert b.sync()["status_bits"] == 0
    b.close()
    net.close()


def test_cvbatch_rejects_invalid_descriptions(mcx):
    probs = _problems()
    d = _desc(probs)
    with pytest.raises(Exception):
        mcx.CVBatch(d, control="learned", net=None)  # the learned control needs a network
    bad = [dict(d[0], t=np.array([0.05, -1.0]))]
    with pytest.raises(Exception):
        mcx.CVBatch(bad, control="taylor")  # horizons must be positive
    bad = [dict(d[2], paths=0)]
    with pytest.raises(Exception):
        mcx.CVBatch(bad, control="none")
    col = d[2]["col"].copy()
    col[5] = 10 ** 6
    with pytest.raises(Exception):
        mcx.CVBatch([dict(d[2], col=col)], control="none")  # column out of range
