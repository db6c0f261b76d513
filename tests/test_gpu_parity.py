"""GPU parity: the CUDA path, called through the C-ABI, against the CPU oracle.

* Preparation tables (rates, potentials, kept columns, alias tables) are
  compared bit for bit.
* Paths are compared bit for bit: end index, jump count, FNV-1a hash of the
  visited indices and the log-weight, in FP32 and FP64, for all three
  functionals (the draw schedule is the same on both sides).
* Per-entry estimates use the same paths, so they differ only in the weight
  exponential and the summation order: FP64 paths agree to 1e-12 relative;
  FP32 paths (FP32 exp, compensated FP32 lane sums) to 2e-6 of the entry's
  absolute scale sum |W v|/M.
* Statistical agreement with exp(tA)v and edge cases (t = 0, no entries,
  isolated nodes, M = 1, invalid CSR).
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
    "grid2d_16": lambda: (W.grid_laplacian_2d(16), 10.0 / (4 * 17 ** 2)),
    "er_2000": lambda: (W.erdos_renyi(2000, 10, 5), 0.09),
    "weighted_120": lambda: (W.dense_to_csr(_conditioned(120, 3)), 1.0),
    "ctmc_500": lambda: (W.random_generator(500, 4), 1.0),
    "ba_3000": lambda: (W.barabasi_albert(3000, 5, 2), 0.05),
}


@pytest.fixture(scope="module", params=sorted(CASES))
def case(request, mcx):
    csr, t = CASES[request.param]()
    plan = mcx.Plan.from_csr(csr)
    og = OW.Graph(csr)
    assert og.status == 0
    yield request.param, csr, t, plan, og
    plan.close()


def test_prep_tables_bit_equal(case):
    name, csr, t, plan, og = case
    ex = {k: v.cpu().numpy() for k, v in plan.export().items()}
    m = og.nnz_off
    assert plan.info()["nnz_off"] == m
    assert np.array_equal(ex["deg"], og.deg)
    assert np.array_equal(ex["row_start"], og.row_start)
    assert np.array_equal(ex["weighted"], og.weighted)
    for k in ("inv_rate32", "delta32", "inv_rate64", "delta64"):
        assert np.array_equal(ex[k].view(np.uint8), getattr(og, k).view(np.uint8)), k
    assert np.array_equal(ex["edge_col"][:m], og.edge_col[:m])
    assert np.array_equal(ex["alias_col"][:m], og.alias_col[:m])
    assert np.array_equal(ex["thresh"][:m].view(np.uint32), og.thresh[:m])


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("mode,nsteps", [("exact", 1), ("strang", 7), ("lie", 3)])
def test_paths_bit_exact(case, prec, mode, nsteps):
    name, csr, t, plan, og = case
    n = csr.n
    for entry in (0, n // 2, n - 1):
        first = 12345 + 1000 * entry
        g = plan.trace(t, entry, seed=77, first_path=first, count=3000, mode=mode, nsteps=nsteps, prec=prec)
        g = {k: v.cpu().numpy() for k, v in g.items()}
        o = og.trace(t, entry, 77, first, 3000, mode=mode, nsteps=nsteps, prec=prec)
        assert np.array_equal(g["end"], o["end"]), (name, entry)
        assert np.array_equal(g["njumps"].view(np.uint32), o["njumps"]), (name, entry)
        assert np.array_equal(g["hash"].view(np.uint64), o["hash"]), (name, entry)
        assert np.array_equal(g["logw"].view(np.uint64), o["logw"].view(np.uint64)), (name, entry)
        assert o["njumps"].max() > 0


def _estimate_both(plan, og, v, t, M, entries, mode="exact", nsteps=1, prec="fp32", seed=3, offset=0):
    ent = None if entries is None else _cuda(entries, torch.int32)
    gm, gs = plan.estimate(_cuda(v, torch.float64), t, M, entries=ent, seed=seed, path_offset=offset, mode=mode,
                           nsteps=nsteps, prec=prec)
    om, os_, _ = og.estimate(v, t, M, entries=entries, seed=seed, path_offset=offset, mode=mode, nsteps=nsteps,
                             prec=prec)
    return gm.cpu().numpy(), gs.cpu().numpy(), om, os_


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_estimates_match_oracle_same_paths(case, prec):
    """Ragged sizes: 333 entries (not a multiple of 8 warps/block), M = 1000 (not a
    multiple of 32 lanes); a second call with 3 entries x 70000 paths exercises the
    multi-chunk reduction."""
    name, csr, t, plan, og = case
    n = csr.n
    v = W.uniform_vector(n, 1, -1.0, 1.0) if name != "ctmc_500" else W.uniform_vector(n, 1)
    rng = np.random.default_rng(0)
    for entries, M in ((np.sort(rng.choice(n, min(333, n - 7), replace=False)).astype(np.int32), 1000),
                       (np.array([0, n // 3, n - 1], np.int32), 70000)):
        gm, gs, om, os_ = _estimate_both(plan, og, v, t, M, entries, prec=prec)
        scale, _, _ = og.estimate(np.abs(v), t, M, entries=entries, seed=3, prec=prec)
        tol = 1e-12 if prec == "fp64" else 2e-6
        assert np.all(np.abs(gm - om) <= tol * scale + 1e-300), (name, np.max(np.abs(gm - om) / scale))
        assert np.allclose(gs, os_, rtol=1e-3 if prec == "fp32" else 1e-9, atol=1e-6 * scale.max())


@pytest.mark.parametrize("vscale", [1e-30, 1e30])
def test_fp32_estimates_at_any_scale_of_v(mcx, vscale):
    """FP32 paths read an exactly scaled copy of v (v times a power of two), so the
    estimates and standard errors of v scaled by 1e-30 or 1e30 match the oracle on the
    same paths as those of v itself do: the squared weights neither underflow (a zero
    standard error) nor overflow (a false overflow flag).  Plain estimates (one and
    several chunks per entry, and the lane layout), the quasi-random estimate and the
    level difference."""
    csr, t = W.erdos_renyi(2000, 10, 5), 0.09
    plan = mcx.Plan.from_csr(csr)
    og = OW.Graph(csr)
    v = W.uniform_vector(2000, 1, -1.0, 1.0) * vscale
    rng = np.random.default_rng(0)
    for entries, M in ((np.sort(rng.choice(2000, 333, replace=False)).astype(np.int32), 1000),
                       (np.array([0, 666, 1999], np.int32), 70000),
                       (np.arange(0, 2000, 5, dtype=np.int32), 40)):
        gm, gs, om, os_ = _estimate_both(plan, og, v, t, M, entries)
        scale, _, _ = og.estimate(np.abs(v), t, M, entries=entries, seed=3)
        assert np.all(np.abs(gm - om) <= 2e-6 * scale), np.max(np.abs(gm - om) / scale)
        assert np.all(gs > 0) and np.allclose(gs, os_, rtol=1e-3, atol=0)
    ent = np.arange(0, 2000, 7, dtype=np.int32)
    qm, _ = plan.estimate_rqmc(_cuda(v, torch.float64), t, 5, 4, entries=_cuda(ent, torch.int32), seed=2)
    oq, _, _ = og.estimate_rqmc(v, t, 5, 4, entries=ent, seed=2)
    qs, _, _ = og.estimate_rqmc(np.abs(v), t, 5, 4, entries=ent, seed=2)
    assert np.all(np.abs(qm.cpu().numpy() - oq) <= 2e-6 * qs)
    dm, ds = plan.estimate_level_difference(_cuda(v, torch.float64), t, 8, 300, entries=_cuda(ent, torch.int32),
                                            seed=3)
    od, os_ = og.estimate_level_difference(v, t, 8, 300, entries=ent, seed=3)
    ow, _, _ = og.estimate(np.abs(v), t, 300, entries=ent, seed=3, mode="strang", nsteps=8)
    assert np.all(np.abs(dm.cpu().numpy() - od) <= 2e-6 * (np.abs(od) + os_ * np.sqrt(300)) + 1e-13 * ow)
    assert np.all(ds.cpu().numpy() > 0)
    assert plan.sync()["status_bits"] == 0
    plan.close()


def test_functionals_estimates_match_oracle(mcx):
    a = _conditioned(50, 9)
    csr = W.dense_to_csr(a)
    plan = mcx.Plan.from_csr(csr)
    og = OW.Graph(csr)
    v = W.uniform_vector(50, 4, 0.2, 1.0)
    for mode, N in (("strang", 2), ("lie", 2), ("strang", 9)):
        for prec in ("fp32", "fp64"):
            gm, gs, om, os_ = _estimate_both(plan, og, v, 2.0, 4000, None, mode=mode, nsteps=N, prec=prec)
            tol = 1e-12 if prec == "fp64" else 2e-6
            assert np.all(np.abs(gm - om) <= tol * np.abs(om)), (mode, prec)
    # and the Strang estimate is unbiased for the Strang product
    gm, gs, _, _ = _estimate_both(plan, og, v, 2.0, 20000, None, mode="strang", nsteps=2, prec="fp32")
    zstats.check((gm - OD.split_expmv(a, 2.0, 2, v, "strang")) / gs, samples=20000)
    plan.close()


def test_grid2d_full_vector_vs_kronecker(mcx):
    """32x32 Dirichlet grid, ~10 jumps per path, 2000 paths per entry, every entry."""
    m = 32
    csr = W.grid_laplacian_2d(m)
    t = 10.0 / (4 * (m + 1) ** 2)
    v = W.uniform_vector(m * m, 0)
    x = OD.grid2d_expmv(m, t, v)
    plan = mcx.Plan.from_csr(csr)
    for prec in ("fp32", "fp64"):
        gm, gs = plan.estimate(_cuda(v, torch.float64), t, 2000, prec=prec)
        zstats.check((gm.cpu().numpy() - x) / gs.cpu().numpy(), samples=2000)
    # centre entry (16, 16) -> 528 with 10^6 paths, seed 0: |z| <= 3
    gm, gs = plan.estimate(_cuda(v, torch.float64), t, 10 ** 6, entries=_cuda([528], torch.int32), seed=0)
    z = (gm.item() - x[528]) / gs.item()
    assert abs(z) <= 3, z
    plan.close()


def test_power_iteration_vs_oracle(mcx):
    csr = W.erdos_renyi(5000, 10, 1)
    lam, it = mcx.power_iteration(_cuda(csr.row_ptr, torch.int64), _cuda(csr.col, torch.int32),
                                  _cuda(csr.val, torch.float64), max_iters=2000, tol=1e-13)
    want = OD.power_iteration(csr.to_scipy(), iters=20000, tol=1e-15)
    assert abs(lam - want) / want < 1e-10, (lam, want, it)
    k = W.dense_to_csr(np.ones((12, 12)) - np.eye(12))
    lam, _ = mcx.power_iteration(_cuda(k.row_ptr, torch.int64), _cuda(k.col, torch.int32),
                                 _cuda(k.val, torch.float64))
    assert abs(lam - 11.0) < 1e-12


@pytest.mark.parametrize("scale", [1.0, 1e-30, 1e60])
def test_power_iteration_fused_rows_at_scale(mcx, scale):
    """A matrix without long rows (the fused one-kernel iteration) with its values
    scaled by 1, 1e-30 and 1e60: the quotient agrees with the oracle's to 1e-10."""
    import dataclasses

    csr = W.erdos_renyi(50000, 10, 4)
    assert np.diff(csr.row_ptr).max() <= 32
    csr = dataclasses.replace(csr, val=csr.val * scale)
    lam, it = mcx.power_iteration(_cuda(csr.row_ptr, torch.int64), _cuda(csr.col, torch.int32),
                                  _cuda(csr.val, torch.float64), max_iters=2000, tol=1e-13)
    want = OD.power_iteration(csr.to_scipy(), iters=20000, tol=1e-15)
    assert abs(lam - want) / want < 1e-10, (lam, want, it)


@pytest.mark.parametrize("scale", [1.0, 1e-30, 1e60])
def test_power_iteration_hub_rows_and_fp64_fallback(mcx, scale):
    """Barabasi-Albert hubs take the warp-per-row kernels; values below 2^-74 or
    above 2^127 are outside the double-float range and take the FP64 kernels."""
    import dataclasses

    import scipy.sparse as sp

    a = W.barabasi_albert(6000, 5, 2).to_scipy().tolil()
    a.resize((6001, 6001))
    a[6000, :6000] = 1.0  # a hub row of 6000 entries: the block-per-row kernel
    a[:6000, 6000] = 1.0
    m = sp.csr_matrix(a)
    m.sort_indices()
    csr = W.CSR(6001, m.indptr.astype(np.int64), m.indices.astype(np.int32), m.data.astype(np.float64))
    deg = np.diff(csr.row_ptr)
    assert deg.max() > 1024 and np.any((deg > 32) & (deg <= 1024))
    csr = dataclasses.replace(csr, val=csr.val * scale)
    lam, it = mcx.power_iteration(_cuda(csr.row_ptr, torch.int64), _cuda(csr.col, torch.int32),
                                  _cuda(csr.val, torch.float64), max_iters=20000, tol=1e-13)
    want = OD.power_iteration(csr.to_scipy(), iters=200000, tol=1e-15)
    assert abs(lam - want) / want < 1e-10, (lam, want, it)


# ---------------------------------------------------------------------------
# Edge cases
# ---------------------------------------------------------------------------

def test_zero_time_returns_v_exactly(mcx):
    csr = W.erdos_renyi(300, 5, 0)
    plan = mcx.Plan.from_csr(csr)
    v = W.uniform_vector(300, 2, -1, 1)
    gm, gs = plan.estimate(_cuda(v, torch.float64), 0.0, 100)
    assert np.array_equal(gm.cpu().numpy(), v) and np.all(gs.cpu().numpy() == 0)
    plan.close()


def test_no_entries_and_single_path(mcx):
    csr = W.erdos_renyi(300, 5, 0)
    plan = mcx.Plan.from_csr(csr)
    og = OW.Graph(csr)
    v = W.uniform_vector(300, 2)
    gm, gs = plan.estimate(_cuda(v, torch.float64), 0.3, 100, entries=torch.empty(0, dtype=torch.int32).cuda())
    assert gm.numel() == 0
    gm, gs, om, _ = _estimate_both(plan, og, v, 0.3, 1, np.arange(300, dtype=np.int32), prec="fp64")
    assert np.allclose(gm, om, rtol=1e-12) and np.all(gs == 0)
    plan.close()


def test_diagonal_and_isolated_nodes_exact(mcx):
    d = np.array([-2.0, 0.0, 0.3, 1.7, -0.5])
    a = np.diag(d)
    a[4, 0] = a[0, 4] = 0.0
    csr = W.dense_to_csr(a)
    plan = mcx.Plan.from_csr(csr)
    v = np.array([1.0, 2.0, -3.0, 0.5, 4.0])
    for prec, tol in (("fp32", 1e-6), ("fp64", 1e-15)):
        gm, gs = plan.estimate(_cuda(v, torch.float64), 0.9, 64, prec=prec)
        want = np.exp(0.9 * d) * v
        assert np.all(np.abs(gm.cpu().numpy() - want) <= tol * np.abs(want))
    plan.close()


@pytest.mark.parametrize("a00", [0.0, -1.25, 0.7])
def test_single_state(mcx, a00):
    """n = 1: no jumps, exp(t a) v exactly for the backward form (any M, both layouts,
    both precisions), the forward form and the total communicability."""
    rp = np.array([0, 1], np.int64) if a00 != 0.0 else np.array([0, 0], np.int64)
    col = np.array([0], np.int32)[: rp[1]]
    val = np.array([a00])[: rp[1]]
    plan = mcx.Plan(_cuda(rp, torch.int64), _cuda(col, torch.int32), _cuda(val, torch.float64))
    t, v = 0.8, np.array([1.5])
    want = math.exp(t * a00) * 1.5
    for M in (1, 40, 5000):
        for prec, tol in (("fp32", 1e-6), ("fp64", 1e-15)):
            gm, gs = plan.estimate(_cuda(v, torch.float64), t, M, prec=prec)
            assert abs(gm.item() - want) <= tol * want and gs.item() == 0.0
    # forward and TC sum 1000 equal FP64 terms: within 1000 * 2^-53 of the value
    x, _ = plan.forward(_cuda(v, torch.float64), t, 1000, prec="fp64")
    assert abs(x.item() - want) <= 2e-13 * want
    tc, se = plan.total_communicability(t, 1000, prec="fp64")
    assert abs(tc.item() - math.exp(t * a00)) <= 2e-13 * math.exp(t * a00) and se.item() == 0.0
    assert plan.sync()["status_bits"] == 0
    plan.close()


def test_zero_potential_gives_one(mcx):
    q = W.random_generator(2000, 7)
    plan = mcx.Plan.from_csr(q)
    gm, gs = plan.estimate(_cuda(np.ones(2000), torch.float64), 2.0, 256)
    assert np.abs(gm.cpu().numpy() - 1.0).max() < 1e-5
    plan.close()


@pytest.mark.parametrize("bad,code", [("unsorted", -1), ("range", -1), ("negoff", -2), ("nan", -3), ("rowptr", -1)])
def test_invalid_csr_rejected(mcx, bad, code):
    a = W.dense_to_csr(_conditioned(10, 3))
    rp, col, val = a.row_ptr.copy(), a.col.copy(), a.val.copy()
    r0, r1 = int(rp[2]), int(rp[3])
    if bad == "unsorted":
        col[r0], col[r0 + 1] = col[r0 + 1], col[r0]
    elif bad == "range":
        col[r1 - 1] = 10
    elif bad == "negoff":
        k = [p for p in range(r0, r1) if col[p] != 2][0]
        val[k] = -0.5
    elif bad == "nan":
        val[r0] = float("nan")
    else:
        rp[5] = rp[6] + 1
    with pytest.raises(mcx.MCXError) as e:
        mcx.Plan(_cuda(rp, torch.int64), _cuda(col, torch.int32), _cuda(val, torch.float64))
    assert e.value.code == code
    og = OW.Graph(W.CSR(10, rp, col, val)) if bad != "rowptr" else None
    if og is not None:
        assert og.status == code


def test_host_input_plan_equals_device_plan(mcx):
    csr = W.erdos_renyi(3000, 8, 9)
    p1 = mcx.Plan.from_csr(csr)
    p2 = mcx.Plan.from_csr(csr, device="cpu")
    v = _cuda(W.uniform_vector(3000, 0), torch.float64)
    a, _ = p1.estimate(v, 0.1, 300)
    b, _ = p2.estimate(v, 0.1, 300)
    assert torch.equal(a, b)
    p1.close()
    p2.close()


def test_deterministic_and_offsets_compose(mcx):
    csr = W.erdos_renyi(4000, 10, 3)
    plan = mcx.Plan.from_csr(csr)
    v = _cuda(W.uniform_vector(4000, 0), torch.float64)
    a, _ = plan.estimate(v, 0.1, 500, seed=5)
    b, _ = plan.estimate(v, 0.1, 500, seed=5)
    assert torch.equal(a, b)
    c, _ = plan.estimate(v, 0.1, 500, seed=6)
    assert not torch.equal(a, c)
    lo, _ = plan.estimate(v, 0.1, 200, seed=5, prec="fp64")
    hi, _ = plan.estimate(v, 0.1, 300, seed=5, path_offset=200, prec="fp64")
    al, _ = plan.estimate(v, 0.1, 500, seed=5, prec="fp64")
    assert torch.allclose((200 * lo + 300 * hi) / 500, al, rtol=1e-12, atol=0)
    plan.close()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_lane_layout_matches_oracle(mcx, prec):
    """At most 64 paths per entry the walker runs one lane per entry: same paths,
    same accumulators, results against the oracle on 1000 ragged entries."""
    csr = W.erdos_renyi(5000, 10, 8)
    plan = mcx.Plan.from_csr(csr)
    og = OW.Graph(csr)
    v = W.uniform_vector(5000, 3, -1.0, 1.0)
    ent = np.sort(np.random.default_rng(1).choice(5000, 1000, replace=False)).astype(np.int32)
    for M in (1, 17, 64):
        gm, gs, om, os_ = _estimate_both(plan, og, v, 0.1, M, ent, prec=prec, seed=M)
        scale, _, _ = og.estimate(np.abs(v), 0.1, M, entries=ent, seed=M, prec=prec)
        tol = 1e-12 if prec == "fp64" else 2e-6
        assert np.all(np.abs(gm - om) <= tol * scale), (M, np.max(np.abs(gm - om) / scale))
        if M > 1:
            assert np.allclose(gs, os_, rtol=1e-3 if prec == "fp32" else 1e-9, atol=1e-6 * scale.max())
    st = plan.sync()
    assert st["paths"] == 1000 * (1 + 17 + 64)
    plan.close()


def test_expm_multiply_host_and_device_buffers(mcx):
    """The one-call C-ABI entry point mcx_expm_multiply: with host arrays (copied in and
    out inside the call) and with device arrays it gives, bit for bit, the estimates of
    a plan's mcx_estimate on the same paths; with t <= 0 it takes beta_scale/lambda_max
    from the same power iteration as mcx_power_iteration; mixed arrays are refused."""
    csr = W.erdos_renyi(3000, 8, 2)
    vh = W.uniform_vector(3000, 4)
    rp, col, val = (torch.as_tensor(x) for x in (csr.row_ptr, csr.col, csr.val))
    ent = torch.as_tensor(W.random_entries(3000, 100, 1))
    v = torch.as_tensor(vh)
    dev = [x.cuda() for x in (rp, col, val, v, ent)]
    hm, hs, t1 = mcx.expm_multiply(rp, col, val, v, t=0.1, paths=500, entries=ent, seed=5)
    dm, ds, _ = mcx.expm_multiply(*dev[:4], t=0.1, paths=500, entries=dev[4], seed=5)
    plan = mcx.Plan(*dev[:3])
    pm, ps = plan.estimate(dev[3], 0.1, 500, entries=dev[4], seed=5)
    assert t1 == 0.1 and not hm.is_cuda and dm.is_cuda
    assert torch.equal(hm, pm.cpu()) and torch.equal(hs, ps.cpu())
    assert torch.equal(dm, pm) and torch.equal(ds, ps)
    lam, _ = mcx.power_iteration(*dev[:3], max_iters=1000, tol=1e-10)
    hm2, _, t2 = mcx.expm_multiply(rp, col, val, v, t=None, beta_scale=0.5, paths=200, seed=1)
    assert t2 == 0.5 / lam
    pm2, _ = plan.estimate(dev[3], t2, 200, seed=1)
    assert torch.equal(hm2, pm2.cpu())
    plan.close()
    with pytest.raises(ValueError):
        mcx.expm_multiply(dev[0], col, val, v, t=0.1)
