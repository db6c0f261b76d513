"""GPU parity of the total-communicability mode TC(t) = 1^T exp(tA) 1 (Sec. 6;
Theorem 2 and Algorithm 2 with v = 1) through the C-ABI.

* The GPU's TC over paths [o, o + M) equals n times the mean path weight of the
  oracle's forward paths with v = 1 over the same paths (same draws: the
  per-path weights are the bit-exact log-weights of the forward trace), to
  1e-12 relative in FP64 and 2e-6 in FP32 (per-path e^L in FP32).
* Statistical: TC against 1^T expm(tA) 1 (dense), and STRANG/LIE against
  1^T (split product) 1, by z-scores over seeds.
* path_offset composes; t = 0 gives n exactly; M < 2 is rejected.
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


def _oracle_tc(csr, t, M, seed, offset=0, mode="exact", nsteps=1, prec="fp32"):
    g = OW.Graph(csr)
    tr = g.forward_trace(np.ones(csr.n), t, seed, offset, M, mode=mode, nsteps=nsteps, prec=prec)
    w = np.exp(tr["logw"])
    return csr.n * w.mean(), csr.n * w.std(ddof=1) / math.sqrt(M)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("mode,nsteps", [("exact", 1), ("strang", 4), ("lie", 3)])
def test_tc_same_paths_as_oracle(mcx, prec, mode, nsteps):
    csr = W.erdos_renyi(2000, 6, 5)  # symmetric: the plan of A is that of A^T
    plan = mcx.Plan.from_csr(csr)
    t = 0.15
    M = 60000  # several warps' chunks and a ragged last chunk
    tc, se = plan.total_communicability(t, M, mode=mode, nsteps=nsteps, seed=13, path_offset=5, prec=prec)
    otc, ose = _oracle_tc(csr, t, M, 13, 5, mode, nsteps, prec)
    tol = 1e-12 if prec == "fp64" else 2e-6
    assert abs(tc.item() - otc) <= tol * otc, (tc.item(), otc)
    assert abs(se.item() - ose) <= (1e-9 if prec == "fp64" else 1e-3) * ose
    plan.close()


def test_tc_weighted_nonsymmetric_rows(mcx):
    """A weighted matrix: the plan is built from A^T, TC = 1^T exp(tA) 1."""
    rng = np.random.default_rng(3)
    n = 120
    a = np.where(rng.random((n, n)) < 0.1, rng.lognormal(0, 0.5, (n, n)), 0.0)
    np.fill_diagonal(a, -0.3)
    b = W.dense_to_csr(a.T)
    plan = mcx.Plan.from_csr(b)
    t = 0.4
    want = float(np.ones(n) @ OD.expm_dense(t * a) @ np.ones(n))
    zs = []
    for seed in range(8):
        tc, se = plan.total_communicability(t, 200000, seed=seed, prec="fp64")
        zs.append((tc.item() - want) / se.item())
    zstats.check(np.array(zs), samples=200000)
    otc, _ = _oracle_tc(b, t, 30000, 1, 0, prec="fp64")
    tc, _ = plan.total_communicability(t, 30000, seed=1, prec="fp64")
    assert abs(tc.item() - otc) <= 1e-12 * otc
    plan.close()


def test_tc_split_modes_vs_split_products(mcx):
    csr = W.erdos_renyi(200, 5, 2)
    a = csr.to_scipy().toarray()
    plan = mcx.Plan.from_csr(csr)
    t, N = 0.3, 2
    for mode in ("strang", "lie"):
        want = float(np.ones(200) @ OD.split_expmv(a, t, N, np.ones(200), mode))
        zs = []
        for seed in range(6):
            tc, se = plan.total_communicability(t, 100000, mode=mode, nsteps=N, seed=100 + seed, prec="fp64")
            zs.append((tc.item() - want) / se.item())
        assert abs(np.mean(zs)) < 5 / math.sqrt(6) and np.max(np.abs(zs)) < 4.5, (mode, zs)
    plan.close()


def test_tc_offset_composes_and_edge_cases(mcx):
    csr = W.erdos_renyi(500, 4, 1)
    plan = mcx.Plan.from_csr(csr)
    t = 0.2
    a, sa = plan.total_communicability(t, 4000, seed=3, path_offset=0, prec="fp64")
    b, sb = plan.total_communicability(t, 4000, seed=3, path_offset=4000, prec="fp64")
    c, _ = plan.total_communicability(t, 8000, seed=3, path_offset=0, prec="fp64")
    assert abs((a.item() + b.item()) / 2 - c.item()) <= 1e-12 * c.item()
    z, sz = plan.total_communicability(0.0, 10, prec="fp64")
    assert z.item() == 500.0 and sz.item() == 0.0
    with pytest.raises(Exception):
        plan.total_communicability(t, 1)
    plan.close()


def test_tc_start_tables_survive_and_refresh(mcx):
    """The plan keeps the start tables of v = 1 between TC calls; a forward call with
    another v replaces them, and the next TC call rebuilds them (same result)."""
    csr = W.erdos_renyi(3000, 5, 8)
    plan = mcx.Plan.from_csr(csr)
    t = 0.25
    a, _ = plan.total_communicability(t, 50000, seed=21, prec="fp64")
    b, _ = plan.total_communicability(t, 50000, seed=21, prec="fp64")
    v = torch.as_tensor(W.uniform_vector(3000, 4)).cuda()
    plan.forward(v, t, 20000, seed=5)
    c, _ = plan.total_communicability(t, 50000, seed=21, prec="fp64")
    assert a.item() == b.item() == c.item()
    otc, _ = _oracle_tc(csr, t, 50000, 21, prec="fp64")
    assert abs(a.item() - otc) <= 1e-12 * otc
    plan.close()
