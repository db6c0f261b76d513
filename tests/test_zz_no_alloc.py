"""mcx_estimate_noalloc: the estimate for callers that cannot allocate device
memory once they are running (a service that reserves its memory at start-up
and must keep it fixed, or a host framework whose pool allocator owns the
device memory).  It must give the same numbers as mcx_estimate, bit for bit,
call after call, while keeping its scratch in the library's fixed device
array, and agree with the oracle on the same paths.

Called straight through the C-ABI (ctypes), with torch only providing device
buffers allocated before the calls.
"""
import ctypes as C

import numpy as np
import pytest

import workloads as W
from oracle import walker as OW

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _p(t):
    return C.c_void_p(t.data_ptr()) if t is not None else C.c_void_p(0)


def _call(L, fn, plan, v, t, M, ent, n_ent, seed, prec, mean, sem):
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return getattr(L, fn)(plan._h, _p(v), float(t), 0, 1, int(M), _p(ent), int(n_ent), int(seed), 0, prec,
                          _p(mean), _p(sem), stream)


@pytest.mark.parametrize("prec", [0, 1])
def test_noalloc_matches_estimate_two_calls_in_a_row(prec):
    import paper_1904_12759_gb300 as P

    L = P.load()
    csr = W.erdos_renyi(3000, 8, 11)
    plan = P.Plan.from_csr(csr)
    vh = W.uniform_vector(3000, 1, -1.0, 1.0)
    v = torch.as_tensor(vh).cuda()
    og = OW.Graph(csr)
    t = 0.12
    tol = 2e-6 if prec == 0 else 1e-12
    # (entries, paths): several chunks per entry, so the fixed scratch array is used;
    # and the full vector with one chunk per entry
    cases = [(torch.tensor([0, 1499, 2999], dtype=torch.int32).cuda(), 70000),
             (torch.arange(0, 3000, 7, dtype=torch.int32).cuda(), 5000),
             (None, 1000)]
    for ent, M in cases:
        n_ent = 3000 if ent is None else ent.numel()
        for call in range(2):
            seed = 40 + call
            ref_m = torch.empty(n_ent, dtype=torch.float64, device="cuda")
            ref_s = torch.empty_like(ref_m)
            got_m = torch.full_like(ref_m, float("nan"))
            got_s = torch.full_like(ref_m, float("nan"))
            assert _call(L, "mcx_estimate", plan, v, t, M, ent, n_ent, seed, prec, ref_m, ref_s) == 0
            assert _call(L, "mcx_estimate_noalloc", plan, v, t, M, ent, n_ent, seed, prec, got_m, got_s) == 0
            torch.cuda.synchronize()
            # same kernels, same chunking, same reduction order: identical numbers
            assert torch.equal(got_m, ref_m) and torch.equal(got_s, ref_s), (M, call)
        # and the oracle's estimate over the same paths (last call's seed)
        ent_np = np.arange(3000, dtype=np.int32) if ent is None else ent.cpu().numpy()
        sel = slice(None) if ent_np.size <= 64 else slice(0, None, ent_np.size // 32)
        om, osd, _ = og.estimate(vh, t, M, entries=ent_np[sel], seed=seed, prec="fp64" if prec else "fp32")
        gm = got_m.cpu().numpy()[sel]
        scale = og.estimate(np.abs(vh), t, M, entries=ent_np[sel], seed=seed, prec="fp64" if prec else "fp32")[0]
        assert np.all(np.abs(gm - om) <= tol * scale), (M, np.max(np.abs(gm - om) / scale))
        assert np.allclose(got_s.cpu().numpy()[sel], osd, rtol=1e-3)
    plan.sync()
    plan.close()


def test_noalloc_rejects_requests_beyond_its_scratch():
    """70000 entries x 2048 paths split into 2 chunks each need 140000 partials, more
    than the 131072 the fixed array holds: rejected before anything runs."""
    import paper_1904_12759_gb300 as P

    L = P.load()
    csr = W.erdos_renyi(70000, 6, 2)
    plan = P.Plan.from_csr(csr)
    v = torch.ones(70000, dtype=torch.float64, device="cuda")
    m = torch.full((70000,), -7.0, dtype=torch.float64, device="cuda")
    s = torch.full_like(m, -7.0)
    ent = torch.arange(70000, dtype=torch.int32, device="cuda")
    rc = _call(L, "mcx_estimate_noalloc", plan, v, 0.1, 2048, ent, 70000, 1, 0, m, s)
    assert rc == -8  # MCX_E_UNSUPPORTED
    torch.cuda.synchronize()
    assert torch.all(m == -7.0)
    # within the limit (one chunk per entry) the same request shape is accepted
    rc = _call(L, "mcx_estimate_noalloc", plan, v, 0.1, 1000, ent, 70000, 1, 0, m, s)
    assert rc == 0
    torch.cuda.synchronize()
    assert torch.all(m >= 1.0 - 1e-5)  # exp(tA)1 >= 1 for A >= 0
    plan.close()
