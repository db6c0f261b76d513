"""GPU parity of the multilevel level difference (mcx_estimate_level_difference)
against the oracle on the same paths, and the multilevel driver.

Both sides walk the same paths with bit-identical log-weights at both step
counts.  The GPU accumulates e^{L_f} v (-expm1(L_c - L_f)); the oracle takes the
plain definition e^{L_f} v - e^{L_c} v in FP64, whose cancellation costs it up
to ~1e-16 e^{L} |v| per path.  So FP32 paths agree within 2e-6 of the level's
scale (|mean| + SE sqrt(M), a bound on the mean |Y|) plus 1e-13 of the plain
estimate of |v|, FP64 paths within 1e-12 of the level's scale plus 1e-13 of it.
"""
import math

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


@pytest.mark.parametrize("mode", ["strang", "lie"])
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_level_difference_matches_oracle(case, mode, prec):
    name, csr, t, plan, og = case
    n = csr.n
    v = W.uniform_vector(n, 1, -1.0, 1.0)
    rng = np.random.default_rng(0)
    for entries, M, N in ((np.sort(rng.choice(n, min(333, n - 7), replace=False)).astype(np.int32), 1000, 8),
                          (np.array([0, n // 3, n - 1], np.int32), 70000, 6)):
        gm, gs = plan.estimate_level_difference(_cuda(v, torch.float64), t, N, M, entries=_cuda(entries, torch.int32),
                                                seed=5, path_offset=77, mode=mode, prec=prec)
        gm, gs = gm.cpu().numpy(), gs.cpu().numpy()
        om, os_ = og.estimate_level_difference(v, t, N, M, entries=entries, seed=5, path_offset=77, mode=mode,
                                               prec=prec)
        sw, _, _ = og.estimate(np.abs(v), t, M, entries=entries, seed=5, path_offset=77, mode=mode, nsteps=N, prec=prec)
        sy = np.abs(om) + os_ * math.sqrt(M)
        tol = 2e-6 if prec == "fp32" else 1e-12
        assert np.all(np.abs(gm - om) <= tol * sy + 1e-13 * sw), (name, np.max(np.abs(gm - om) / sy))
        assert np.all(np.abs(gs - os_) <= (1e-3 if prec == "fp32" else 1e-9) * os_ + 1e-13 * sw)
    assert plan.sync()["status_bits"] == 0


@pytest.mark.parametrize("mode", ["strang", "lie"])
def test_levels_telescope_on_gpu(mcx, mode):
    """estimate(N_0) + differences at N_1..N_L on the same paths = estimate(N_L)."""
    csr = W.dense_to_csr(_weighted(80, 7))
    plan = mcx.Plan.from_csr(csr)
    v = _cuda(W.uniform_vector(csr.n, 4), torch.float64)
    M, n0, L = 20000, 2, 4
    total, _ = plan.estimate(v, 0.8, M, seed=9, path_offset=3, mode=mode, nsteps=n0)
    total = total.clone()
    for lvl in range(1, L + 1):
        d, _ = plan.estimate_level_difference(v, 0.8, n0 << lvl, M, seed=9, path_offset=3, mode=mode)
        total += d
    fine, _ = plan.estimate(v, 0.8, M, seed=9, path_offset=3, mode=mode, nsteps=n0 << L)
    scale, _ = plan.estimate(v.abs(), 0.8, M, seed=9, path_offset=3, mode=mode, nsteps=n0 << L)
    err = ((total - fine).abs() / scale).max().item()
    assert err < 4e-6, err
    plan.close()


def test_level_difference_edge_cases(mcx):
    csr = W.erdos_renyi(300, 6, 2)
    plan = mcx.Plan.from_csr(csr)
    v = _cuda(W.uniform_vector(csr.n, 3), torch.float64)
    m, s = plan.estimate_level_difference(v, 0.0, 4, 100)
    assert torch.all(m == 0) and torch.all(s == 0)
    for mode, N in (("exact", 4), ("strang", 5), ("lie", 0)):
        with pytest.raises(mcx.MCXError) as e:
            plan.estimate_level_difference(v, 0.1, N, 100, mode=mode)
        assert e.value.code == -1
    m, s = plan.estimate_level_difference(v, 0.1, 4, 100, entries=_cuda([0, csr.n, 2], torch.int32))
    mc = m.cpu().numpy()
    assert np.isnan(mc[1]) and np.all(np.isfinite(mc[[0, 2]]))
    with pytest.raises(mcx.MCXError):
        plan.sync()
    plan.close()


def test_multilevel_driver_against_split_product(mcx):
    from paper_1904_12759_gb300 import mlmc

    csr = W.dense_to_csr(_weighted(80, 11))
    a = csr.to_scipy().toarray()
    plan = mcx.Plan.from_csr(csr)
    v = W.uniform_vector(csr.n, 6)
    t, n0, L = 0.8, 2, 4
    target = OD.split_expmv(a, t, n0 << L, v, "strang")
    mean, sem, levels = mlmc.estimate(plan, _cuda(v, torch.float64), t, n0, L, [200000, 40000, 20000, 10000, 5000],
                                      seed=4)
    zstats.check((mean.cpu().numpy() - target) / sem.cpu().numpy(), samples=5000)
    # the level variances fall with the level (coupled differences)
    V = [float((s.cpu().numpy() ** 2).mean()) * M for (_, s), M in zip(levels, [200000, 40000, 20000, 10000, 5000])]
    assert V[1] < V[0] and V[4] < V[1]
    plan.close()


def test_combine_levels_on_the_device(mcx):
    """mcx_combine_levels: the level means added in level order (bit for bit the same
    sequential FP64 sum) and the standard errors in quadrature."""
    rng = np.random.default_rng(0)
    L, n = 5, 777
    ms = [rng.normal(size=n) for _ in range(L)]
    ss = [rng.uniform(0, 1, n) for _ in range(L)]
    plan = mcx.Plan.from_csr(W.erdos_renyi(10, 2, 1))
    m, s = plan.combine_levels([_cuda(x, torch.float64) for x in ms], [_cuda(x, torch.float64) for x in ss])
    want = ms[0].copy()
    for x in ms[1:]:
        want = want + x
    assert np.array_equal(m.cpu().numpy(), want)
    assert np.allclose(s.cpu().numpy(), np.sqrt(sum(x * x for x in ss)), rtol=1e-15, atol=0)
    with pytest.raises(ValueError):
        plan.combine_levels([_cuda(ms[0], torch.float64)], [])
    plan.close()
