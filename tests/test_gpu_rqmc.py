"""GPU parity of the randomised quasi-Monte Carlo estimator (mcx_estimate_rqmc)
against the oracle on the same scrambled Sobol' points and Philox draws.

Both sides walk the same paths (the quasi-random words are bit-identical), so the
replicate means differ only in the weight exponential and the summation order:
FP64 paths agree to 1e-12 of the entry's absolute scale (the estimate of
|W v|), FP32 paths (FP32 exp, compensated FP32 lane sums) to 2e-6 of it.  The
standard error comes from the spread of the replicate means, so it inherits
that difference once per replicate: |dse| <= 4e-6 scale (FP32), 1e-12 scale
(FP64), besides 1e-9 relative.

Ragged sizes: 333 entries, replicate counts that are not powers of two, 32-point
replicates (one pass of the lanes), 8192-point replicates cut into slices over
several warps, and one-point replicates.
"""
import numpy as np
import pytest

import workloads as W
import zstats
from oracle import dense as OD
from oracle import walker as OW

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def mcx():
    import paper_1904_12759_gb300 as P

    P.load()
    return P


def _cuda(a, dtype):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype).cuda()


def _weighted(n, seed):
    rng = np.random.default_rng(seed)
    a = np.where(rng.random((n, n)) < 0.3, rng.lognormal(0, 1, (n, n)), 0.0)
    np.fill_diagonal(a, 0.0)
    a *= 1.5 / a.sum(axis=1).mean()
    np.fill_diagonal(a, rng.normal(0, 1, n) - a.sum(axis=1))
    return a


CASES = {
    "er_2000": lambda: (W.erdos_renyi(2000, 10, 5), 0.09),
    "weighted_120": lambda: (W.dense_to_csr(_weighted(120, 3)), 1.0),
    "ba_3000": lambda: (W.barabasi_albert(3000, 5, 2), 0.05),
}


@pytest.fixture(scope="module", params=sorted(CASES))
def case(request, mcx):
    csr, t = CASES[request.param]()
    plan = mcx.Plan.from_csr(csr)
    og = OW.Graph(csr)
    yield request.param, csr, t, plan, og
    plan.close()


def _both(plan, og, v, t, log2q, R, entries, mode="exact", nsteps=1, prec="fp32", seed=11):
    ent = None if entries is None else _cuda(entries, torch.int32)
    gm, gs = plan.estimate_rqmc(_cuda(v, torch.float64), t, log2q, R, entries=ent, seed=seed, mode=mode,
                                nsteps=nsteps, prec=prec)
    om, os_, _ = og.estimate_rqmc(v, t, log2q, R, entries=entries, seed=seed, mode=mode, nsteps=nsteps, prec=prec)
    scale, _, _ = og.estimate_rqmc(np.abs(v), t, log2q, R, entries=entries, seed=seed, mode=mode, nsteps=nsteps,
                                   prec=prec)
    return gm.cpu().numpy(), gs.cpu().numpy(), om, os_, scale


def _check(gm, gs, om, os_, scale, prec, label):
    tol, stol = (1e-12, 1e-12) if prec == "fp64" else (2e-6, 4e-6)
    assert np.all(np.abs(gm - om) <= tol * scale + 1e-300), (label, np.max(np.abs(gm - om) / scale))
    assert np.all(np.abs(gs - os_) <= 1e-9 * os_ + stol * scale + 1e-300), (label, np.max(np.abs(gs - os_) / scale))


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_rqmc_matches_oracle(case, prec):
    name, csr, t, plan, og = case
    n = csr.n
    v = W.uniform_vector(n, 1, -1.0, 1.0)
    rng = np.random.default_rng(0)
    ragged = np.sort(rng.choice(n, min(333, n - 7), replace=False)).astype(np.int32)
    for entries, log2q, R in ((ragged, 5, 6), (np.array([0, n // 3, n - 1], np.int32), 13, 4),
                              (ragged[:50], 0, 64)):
        gm, gs, om, os_, scale = _both(plan, og, v, t, log2q, R, entries, prec=prec)
        _check(gm, gs, om, os_, scale, prec, (name, log2q, R))
    st = plan.sync()
    assert st["status_bits"] == 0


@pytest.mark.parametrize("mode,nsteps", [("strang", 5), ("lie", 3)])
def test_rqmc_split_functionals_match_oracle(mcx, mode, nsteps):
    csr = W.dense_to_csr(_weighted(80, 7))
    plan = mcx.Plan.from_csr(csr)
    og = OW.Graph(csr)
    v = W.uniform_vector(csr.n, 4)
    for prec in ("fp32", "fp64"):
        gm, gs, om, os_, scale = _both(plan, og, v, 0.8, 6, 5, None, mode=mode, nsteps=nsteps, prec=prec)
        _check(gm, gs, om, os_, scale, prec, (mode, prec))
    plan.close()


def test_rqmc_edge_cases(mcx):
    csr = W.erdos_renyi(500, 6, 1)
    plan = mcx.Plan.from_csr(csr)
    v = _cuda(W.uniform_vector(csr.n, 3), torch.float64)
    # t = 0 returns v exactly with a zero standard error
    m, s = plan.estimate_rqmc(v, 0.0, 4, 8)
    assert torch.equal(m, v) and torch.all(s == 0)
    # no entries: nothing to do
    e0 = torch.empty(0, dtype=torch.int32, device="cuda")
    m, s = plan.estimate_rqmc(v, 0.1, 4, 8, entries=e0)
    assert m.numel() == 0
    # one replicate: a mean without a standard error
    m, s = plan.estimate_rqmc(v, 0.1, 6, 1, entries=_cuda([3, 4], torch.int32))
    assert torch.all(s == 0) and torch.all(torch.isfinite(m))
    # invalid arguments are rejected at the call
    for log2q, R in ((25, 8), (4, 0), (2, (1 << 16) + 1)):
        with pytest.raises(mcx.MCXError) as e:
            plan.estimate_rqmc(v, 0.1, log2q, R)
        assert e.value.code == -1  # MCX_E_INVALID
    assert plan.sync()["status_bits"] == 0
    # an entry outside [0, n): NaN for it, the others computed, the error at sync
    ent = _cuda([1, csr.n + 5, 2], torch.int32)
    m, s = plan.estimate_rqmc(v, 0.1, 4, 8, entries=ent)
    mc = m.cpu().numpy()
    assert np.isnan(mc[1]) and np.all(np.isfinite(mc[[0, 2]]))
    with pytest.raises(mcx.MCXError) as e:
        plan.sync()
    assert e.value.code == -1
    plan.close()


def test_rqmc_reduces_variance_on_gpu(mcx):
    """Same paths per entry (16 x 2^7): the quasi-random standard errors, which
    the parity above ties to the spread of the replicate means, are below the
    plain estimator's, and both are consistent with expm."""
    csr = W.erdos_renyi(2000, 10, 5)
    plan = mcx.Plan.from_csr(csr)
    t = 0.09
    v = np.ones(csr.n)
    ent = np.arange(0, csr.n, 7, dtype=np.int32)
    x = OD.expmv_dense(csr.to_scipy().toarray(), t, v)[ent]
    vd = _cuda(v, torch.float64)
    q, qs = plan.estimate_rqmc(vd, t, 7, 16, entries=_cuda(ent, torch.int32), seed=2)
    p, ps = plan.estimate(vd, t, 16 << 7, entries=_cuda(ent, torch.int32), seed=2)
    q, qs, p, ps = (a.cpu().numpy() for a in (q, qs, p, ps))
    assert np.mean(qs ** 2) < 0.5 * np.mean(ps ** 2), (np.mean(qs ** 2), np.mean(ps ** 2))
    zstats.check((q - x) / qs, samples=16, dof=15)  # SE from 16 replicate means
    plan.close()


def test_rqmc_replicate_ranges_shard(mcx):
    """Replicates 0..6 and 7..11 as two calls (two ranks) against the oracle with the
    same offsets, and merged by the shard formula against one call over all 12."""
    from paper_1904_12759_gb300 import shard

    csr = W.erdos_renyi(2000, 10, 5)
    plan = mcx.Plan.from_csr(csr)
    og = OW.Graph(csr)
    v = W.uniform_vector(csr.n, 2)
    vd = _cuda(v, torch.float64)
    ent = np.arange(0, csr.n, 13, dtype=np.int32)
    ed = _cuda(ent, torch.int32)
    parts = []
    for r0, R in ((0, 7), (7, 5)):
        gm, gs = plan.estimate_rqmc(vd, 0.09, 6, R, entries=ed, seed=8, replicate_offset=r0)
        om, os_, _ = og.estimate_rqmc(v, 0.09, 6, R, entries=ent, seed=8, replicate_offset=r0)
        _check(gm.cpu().numpy(), gs.cpu().numpy(), om, os_, np.abs(om), "fp32", r0)
        parts.append((gm.cpu().numpy(), gs.cpu().numpy(), R))
    am, asem = plan.estimate_rqmc(vd, 0.09, 6, 12, entries=ed, seed=8)
    mm, ss = shard.merge(np.stack([p[0] for p in parts]), np.stack([p[1] for p in parts]), np.array([7, 5]))
    am, asem = am.cpu().numpy(), asem.cpu().numpy()
    assert np.allclose(mm, am, rtol=4e-6) and np.allclose(ss, asem, rtol=1e-3, atol=1e-6 * np.abs(am).max())
    with pytest.raises(mcx.MCXError):
        plan.estimate_rqmc(vd, 0.09, 6, 12, entries=ed, replicate_offset=0xFFFFFFFF - 5)
    plan.close()
