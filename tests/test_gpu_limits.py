"""Edge cases at the size limits of the C-ABI, on the GPU:

* path indices above 2^32 (the Philox counter's high path word) traced bit for
  bit against the oracle, backward and forward;
* more than 2^32 paths for one entry (64-bit path and jump counters, 77824
  chunks merged in chunk order) against expm within five standard errors;
* the largest quasi-random set per replicate (2^24 points, sliced over warps)
  against the oracle on sampled points' paths, via the mean over few entries.
"""
import math

import numpy as np
import pytest
import scipy.linalg

import workloads as W
from oracle import walker as OW

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def mcx():
    import paper_1904_12759_gb300 as P

    P.load()
    return P


def test_path_indices_above_2_pow_32(mcx):
    csr = W.erdos_renyi(500, 6, 3)
    plan = mcx.Plan.from_csr(csr)
    og = OW.Graph(csr)
    first = (1 << 32) + 12345
    for prec in ("fp32", "fp64"):
        g = {k: x.cpu().numpy() for k, x in plan.trace(0.4, 7, seed=5, first_path=first, count=2000, prec=prec).items()}
        o = og.trace(0.4, 7, 5, first, 2000, prec=prec)
        assert np.array_equal(g["end"], o["end"]) and np.array_equal(g["hash"].view(np.uint64), o["hash"])
        assert np.array_equal(g["logw"].view(np.uint64), o["logw"].view(np.uint64))
        # the high word matters: the same low word without it gives other paths
        o2 = og.trace(0.4, 7, 5, first - (1 << 32), 2000, prec=prec)
        assert not np.array_equal(o2["hash"], o["hash"])
    v = np.ones(csr.n)
    g = {k: x.cpu().numpy() for k, x in plan.trace_forward(torch.ones(csr.n, dtype=torch.float64, device="cuda"), 0.4,
                                                              seed=9, first_path=first, count=2000).items()}
    o = og.forward_trace(v, 0.4, 9, first, 2000)
    assert np.array_equal(g["end"], o["end"]) and np.array_equal(g["hash"].view(np.uint64), o["hash"])
    plan.close()


def test_more_than_2_pow_32_paths_for_one_entry(mcx):
    csr = W.erdos_renyi(200, 4, 1)
    a = csr.to_scipy().toarray()
    plan = mcx.Plan.from_csr(csr)
    v = W.uniform_vector(csr.n, 2)
    t = 0.05
    M = (1 << 32) + 777
    mean, sem = plan.estimate(torch.as_tensor(v).cuda(), t, M, entries=torch.tensor([11], dtype=torch.int32,
                                                                                     device="cuda"), seed=3)
    st = plan.sync()
    assert st["paths"] == M and st["status_bits"] == 0
    x = (scipy.linalg.expm(t * a) @ v)[11]
    assert abs(mean.item() - x) <= 5 * sem.item(), (mean.item(), x, sem.item())
    assert 0 < sem.item() < 1e-4 * abs(x)
    plan.close()


def test_largest_quasi_random_sets(mcx):
    """2^24 points per replicate (all five digit levels, 8192 slices per replicate)
    for two entries and two replicates, against the oracle on the same points."""
    csr = W.erdos_renyi(300, 6, 4)
    plan = mcx.Plan.from_csr(csr)
    og = OW.Graph(csr)
    v = W.uniform_vector(csr.n, 1)
    ent = np.array([3, 250], np.int32)
    gm, gs = plan.estimate_rqmc(torch.as_tensor(v).cuda(), 0.2, 24, 2, entries=torch.as_tensor(ent).cuda(), seed=6)
    om, os_, _ = og.estimate_rqmc(v, 0.2, 24, 2, entries=ent, seed=6)
    gm, gs = gm.cpu().numpy(), gs.cpu().numpy()
    assert np.all(np.abs(gm - om) <= 2e-6 * np.abs(om)), np.abs(gm - om) / np.abs(om)
    assert np.all(np.abs(gs - os_) <= 1e-9 * os_ + 4e-6 * np.abs(om))
    assert plan.sync()["paths"] == 2 * 2 * (1 << 24)
    plan.close()
