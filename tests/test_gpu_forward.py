"""GPU parity of the forward form (Lemma 2, Theorem 2, Algorithm 2) through the C-ABI.

* Forward paths (start draw from the two-level table, walk, end) bit-exact
  against the oracle in FP32 and FP64.
* Estimates on the same paths: exact integer deposits for zero-potential
  plans (CTMC generators) agree to 1e-12; FP64 atomic sums to 1e-12 (FP64,
  summation order) and 2e-6 (FP32 weights).
* Conservation: for a generator every path deposits V somewhere, so
  sum_i x_i = V.
* Statistics against exp(t Q^T) p0 and against exp(tA)v for a non-symmetric A.
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


def _conditioned(n, seed, rate=1.5, dsd=1.0):
    rng = np.random.default_rng(seed)
    a = np.where(rng.random((n, n)) < 0.3, rng.lognormal(0, 1, (n, n)), 0.0)
    np.fill_diagonal(a, 0.0)
    a *= rate / a.sum(axis=1).mean()
    np.fill_diagonal(a, rng.normal(0, dsd, n) - a.sum(axis=1) + rng.normal(0, dsd, n))
    return a


CASES = {
    # (plan matrix B = A^T, v, t); ctmc: B = Q, so x = exp(t Q^T) p0
    "ctmc_3000": lambda: (W.random_generator(3000, 5), W.dirichlet_probability(3000, 1), 1.0),
    "weighted_150": lambda: (W.dense_to_csr(_conditioned(150, 4).T), W.uniform_vector(150, 2), 1.0),
    "er_5000": lambda: (W.erdos_renyi(5000, 8, 3), W.uniform_vector(5000, 3), 0.1),
}


@pytest.fixture(scope="module", params=sorted(CASES))
def fcase(request, mcx):
    b, v, t = CASES[request.param]()
    plan = mcx.Plan.from_csr(b)
    og = OW.Graph(b)
    yield request.param, b, v, t, plan, og
    plan.close()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("mode,nsteps", [("exact", 1), ("strang", 5)])
def test_forward_paths_bit_exact(fcase, prec, mode, nsteps):
    name, b, v, t, plan, og = fcase
    g = plan.trace_forward(_cuda(v, torch.float64), t, seed=11, first_path=777, count=5000, mode=mode,
                           nsteps=nsteps, prec=prec)
    g = {k: x.cpu().numpy() for k, x in g.items()}
    o = og.forward_trace(v, t, 11, 777, 5000, mode=mode, nsteps=nsteps, prec=prec)
    assert np.array_equal(g["start"], o["start"]), name
    assert np.array_equal(g["end"], o["end"]), name
    assert np.array_equal(g["njumps"].view(np.uint32), o["njumps"]), name
    assert np.array_equal(g["hash"].view(np.uint64), o["hash"]), name
    assert np.array_equal(g["logw"].view(np.uint64), o["logw"].view(np.uint64)), name


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_forward_estimates_match_oracle(fcase, prec):
    name, b, v, t, plan, og = fcase
    M = 200003  # not a multiple of anything
    gx, gs = plan.forward(_cuda(v, torch.float64), t, M, seed=4, path_offset=9, prec=prec)
    gx, gs = gx.cpu().numpy(), gs.cpu().numpy()
    ox, os_, _ = og.forward(v, t, M, seed=4, path_offset=9, prec=prec)
    tol = 1e-12 if (prec == "fp64" or name == "ctmc_3000") else 2e-6
    scale = np.abs(ox).max()
    assert np.all(np.abs(gx - ox) <= tol * np.abs(ox) + 1e-13 * scale), (name, np.abs(gx - ox).max())
    assert np.allclose(gs, os_, rtol=1e-6, atol=1e-9 * scale)
    plan.sync()


def test_forward_ctmc_conserves_probability_and_matches_transient(mcx):
    q = W.random_generator(2000, 8)
    p0 = W.dirichlet_probability(2000, 2)
    plan = mcx.Plan.from_csr(q)
    og = OW.Graph(q)
    V = og.start_table(p0)[1]["V"]
    for t in (0.1, 1.0, 10.0):
        x, sem = plan.forward(_cuda(p0, torch.float64), t, 2_000_000, seed=1)
        x, sem = x.cpu().numpy(), sem.cpu().numpy()
        assert abs(x.sum() - V) <= 1e-12 * V  # every path deposits V
        want = OD.uniformization_expmv(q.to_scipy().T.tocsr(), t, p0)
        ok = sem > 0
        zstats.check((x[ok] - want[ok]) / sem[ok], samples=2_000_000)
    plan.sync()
    plan.close()


def test_forward_nonsymmetric_vs_expm(mcx):
    a = _conditioned(40, 12)
    v = W.uniform_vector(40, 5)
    plan = mcx.Plan.from_csr(W.dense_to_csr(a.T))
    x, sem = plan.forward(_cuda(v, torch.float64), 1.0, 4_000_000, seed=2)
    zstats.check((x.cpu().numpy() - OD.expmv_dense(a, 1.0, v)) / sem.cpu().numpy(), samples=4_000_000)
    plan.close()


def test_forward_edge_cases(mcx):
    q = W.random_generator(1500, 3)
    plan = mcx.Plan.from_csr(q)
    p0 = _cuda(W.dirichlet_probability(1500, 4), torch.float64)
    x, sem = plan.forward(p0, 0.0, 1000)
    assert torch.equal(x, p0) and torch.all(sem == 0)
    bad = p0.clone()
    bad[7] = -1.0
    x, _ = plan.forward(bad, 1.0, 1000)
    with pytest.raises(mcx.MCXError) as e:
        plan.sync()
    assert e.value.code == -4
    assert torch.all(torch.isnan(x))
    x, _ = plan.forward(torch.zeros(1500, dtype=torch.float64, device="cuda"), 1.0, 1000)
    with pytest.raises(mcx.MCXError):
        plan.sync()
    plan.close()
