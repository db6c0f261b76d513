"""Parity at the benchmark sizes, in the launch configuration bench.py times, on
sampled outputs the oracle computes one by one (paths are a function of
(seed, entry, path index) only, so the oracle reproduces any sampled entry of a
full-size run):

* Erdos-Renyi n = 1e6, mean degree 10, beta = 1/lambda_max, v = 1, every entry
  x 1000 paths (the default benchmark step): 24 sampled entries; the same graph
  with 16 quasi-random replicates x 64 points per entry: 24 sampled entries.
* 3D heat, 128^3 grid, 4096 entries x 1e6 paths: 2 sampled entries.
* Barabasi-Albert n = 4e6 with the Taylor-only control variate, every entry x
  1 path (the control-variate benchmark at M = 1): 64 sampled entries.
* Total communicability on the small-world graph n = 1e6 at M = 1e6, STRANG
  N = 32: the whole sum over the same paths.
* The 256-generator CTMC batch in one persistent graph launch: the 6 pairs of
  the two smallest generators, exact counts.

FP32 paths: means within 2e-6 of each entry's absolute scale (the path
log-weights are bit-exact; see the parity bar of the small cases), control-variate
residuals within 1e-5 of the entry's scale.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import walker as OW

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def mcx():
    import paper_1904_12759_gb300 as P

    P.load()
    return P


def _dev(csr):
    return [torch.as_tensor(a).cuda() for a in (csr.row_ptr, csr.col, csr.val)]


def test_erdos_renyi_benchmark_step_sampled(mcx):
    csr = W.erdos_renyi(10 ** 6, 10, 0)
    rp, col, val = _dev(csr)
    lam, _ = mcx.power_iteration(rp, col, val, max_iters=1000, tol=1e-10)
    plan = mcx.Plan(rp, col, val)
    v = torch.ones(csr.n, dtype=torch.float64, device="cuda")
    M = 1000
    mean, sem = plan.estimate(v, 1.0 / lam, M, seed=7)  # all entries, the benchmark's launch
    st = plan.sync()
    assert st["status_bits"] == 0 and st["paths"] == csr.n * M
    ent = W.random_entries(csr.n, 24, 3)
    om, osem, _ = OW.Graph(csr).estimate(np.ones(csr.n), 1.0 / lam, M, entries=ent, seed=7)
    gm, gs = mean.cpu().numpy()[ent], sem.cpu().numpy()[ent]
    scale = np.abs(om) + osem * math.sqrt(M)  # >= sum |W v| / M
    assert np.all(np.abs(gm - om) <= 2e-6 * scale), np.max(np.abs(gm - om) / scale)
    assert np.allclose(gs, osem, rtol=1e-3)
    plan.close()


def test_erdos_renyi_rqmc_sampled(mcx):
    """The quasi-random study's launch at M = 1024 (16 replicates x 64 points) over
    every entry: 24 sampled entries against the oracle on the same points."""
    csr = W.erdos_renyi(10 ** 6, 10, 0)
    rp, col, val = _dev(csr)
    lam, _ = mcx.power_iteration(rp, col, val, max_iters=1000, tol=1e-10)
    plan = mcx.Plan(rp, col, val)
    v = torch.ones(csr.n, dtype=torch.float64, device="cuda")
    mean, sem = plan.estimate_rqmc(v, 1.0 / lam, 6, 16, seed=13)
    st = plan.sync()
    assert st["status_bits"] == 0 and st["paths"] == csr.n * 1024
    ent = W.random_entries(csr.n, 24, 5)
    om, osem, _ = OW.Graph(csr).estimate_rqmc(np.ones(csr.n), 1.0 / lam, 6, 16, entries=ent, seed=13)
    gm, gs = mean.cpu().numpy()[ent], sem.cpu().numpy()[ent]
    assert np.all(np.abs(gm - om) <= 2e-6 * np.abs(om)), np.max(np.abs(gm - om) / np.abs(om))
    assert np.all(np.abs(gs - osem) <= 1e-9 * osem + 4e-6 * np.abs(om))
    plan.close()


def test_heat3d_benchmark_sampled(mcx):
    m = 128
    csr = W.grid_laplacian_3d(m)
    t = 20.0 / (6.0 * (m + 1) ** 2)
    v = W.gaussian_bump_3d(m, 0)
    ent = W.random_entries(csr.n, 4096, 0)
    plan = mcx.Plan.from_csr(csr)
    M = 10 ** 6
    mean, sem = plan.estimate(torch.as_tensor(v).cuda(), t, M, entries=torch.as_tensor(ent).cuda(), seed=11)
    pick = np.array([17, 3001])
    om, osem, _ = OW.Graph(csr).estimate(v, t, M, entries=ent[pick], seed=11)
    gm, gs = mean.cpu().numpy()[pick], sem.cpu().numpy()[pick]
    scale = np.abs(om) + osem * math.sqrt(M)
    assert np.all(np.abs(gm - om) <= 2e-6 * scale), np.max(np.abs(gm - om) / scale)
    assert np.allclose(gs, osem, rtol=1e-3)
    plan.close()


def test_barabasi_albert_control_variate_sampled(mcx):
    csr = W.barabasi_albert(4 * 10 ** 6, 5, 0)
    rp, col, val = _dev(csr)
    lam, _ = mcx.power_iteration(rp, col, val, max_iters=20000, tol=1e-9)
    t = 0.5 / lam
    v = W.uniform_vector(csr.n, 0)
    vd = torch.as_tensor(v).cuda()
    plan = mcx.Plan(rp, col, val)
    T, F = mcx.cv_prepare(rp, col, val, vd, t)
    coef = mcx.cv_coefficients(rp, col, val, T, None, t)
    mean, sem = plan.estimate_cv(coef, t, 1, seed=5)  # every entry, one path: the lane layout
    cg = coef.cpu().numpy()
    n = csr.n
    ab = cg[:2 * n].reshape(n, 2)
    ent = W.random_entries(n, 64, 9)
    om, _ = OW.Graph(csr).estimate_cv(ab[:, 0].copy(), ab[:, 1].copy(), cg[2 * n:].copy(), t, 1, entries=ent, seed=5)
    gm = mean.cpu().numpy()[ent]
    scale = np.abs(cg[2 * n:][ent]) + np.abs(om - cg[2 * n:][ent])
    assert np.all(np.abs(gm - om) <= 1e-5 * scale), np.max(np.abs(gm - om) / scale)
    plan.close()


def test_total_communicability_paper_setting(mcx):
    csr = W.small_world(10 ** 6, 1, 0.2, 0)
    plan = mcx.Plan.from_csr(csr)
    M = 10 ** 6
    tc, se = plan.total_communicability(1.0, M, mode="strang", nsteps=32, seed=3)
    tr = OW.Graph(csr).forward_trace(np.ones(csr.n), 1.0, 3, 0, M, mode="strang", nsteps=32, prec="fp32")
    w = np.exp(tr["logw"])
    otc = csr.n * w.mean()
    assert abs(tc.item() - otc) <= 2e-6 * otc, (tc.item(), otc)
    assert abs(se.item() - csr.n * w.std(ddof=1) / math.sqrt(M)) <= 1e-3 * se.item()
    plan.close()


def test_ctmc_batch_benchmark_sampled(mcx):
    """The 256-generator batch of the CTMC benchmark in its persistent graph launch: the
    pairs of the two smallest generators at every horizon against the oracle's
    single-problem forward runs (path indices k * 2^40 + p), count for count."""
    probs = W.ctmc_batch(256, 0)
    b = mcx.Batch(probs)
    b.run(seed=41)
    torch.cuda.synchronize()
    st = b.sync()
    assert st["status_bits"] == 0
    order = sorted(range(len(probs)), key=lambda i: probs[i]["csr"].n)[:2]
    for i in order:
        p = probs[i]
        og = OW.Graph(p["csr"])
        for ti, t in enumerate(p["times"]):
            k = sum(len(q["times"]) for q in probs[:i]) + ti  # pairs numbered problem by problem
            x, _ = b.result(i, ti)
            ox, _, _ = og.forward(p["v"], t, p["paths"], seed=41, path_offset=k << 40)
            assert np.allclose(x.cpu().numpy(), ox, rtol=1e-12, atol=1e-15), (i, ti)
    b.close()
