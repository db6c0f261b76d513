"""Failure paths of the library, made on the host or with a bounded device wait
(nothing here faults, traps or hangs a GPU).

* Allocation failure: the library's test hook makes its k-th device allocation
  from now fail (pool or cudaMalloc).  For every entry point that allocates,
  k = 1, 2, ... fails each of its allocations in turn: the call returns
  MCX_E_OOM, the library's pool usage is back where it was and no cudaMalloc'd
  memory is left behind; once k passes the call's allocations it succeeds.
* Bounded wait: the tensor-core inference's and gradient's MMA waits given a
  limit of zero polls give up at once; the kernel latches the error, drains its
  MMAs with the normal limit, frees its tensor memory and returns: mcx_mlp_sync
  reports MCX_E_TIMEOUT and the context stays usable (a later call is correct).
"""
import numpy as np
import pytest

import workloads as W
from oracle import cv as CV

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

OOM = -6


@pytest.fixture(scope="module")
def mcx():
    import paper_1904_12759_gb300 as P

    P.load()
    return P


def _free_bytes():
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def _oom_sweep(mcx, call, cleanup=lambda r: None, max_k=64):
    """Fail allocation k = 1, 2, ... of `call` until it succeeds; return the number of
    allocations it made.  After each failure: MCX_E_OOM, pool usage and free device
    memory as before the call."""
    from paper_1904_12759_gb300 import MCXError

    cleanup(call())  # warm: torch's caching allocator holds the outputs' memory from now on
    used0 = mcx.debug_pool_usage()[0]
    free0 = _free_bytes()
    for k in range(1, max_k):
        mcx.debug_fail_alloc(k)
        try:
            res = call()
        except MCXError as exc:
            assert exc.code == OOM, (k, exc)
            assert mcx.debug_pool_usage()[0] == used0, k
            assert abs(_free_bytes() - free0) <= 2 << 20, (k, free0 - _free_bytes())
            continue
        finally:
            mcx.debug_fail_alloc(0)
        cleanup(res)
        torch.cuda.synchronize()
        assert mcx.debug_pool_usage()[0] == used0
        return k - 1
    raise AssertionError("the call never succeeded")


def _close(obj):
    if obj is not None:
        obj.close()


def test_allocation_failure_every_entry_point(mcx, tmp_path):
    er = W.erdos_renyi(3000, 8, 2)
    wt = W.dense_to_csr(np.where(np.random.default_rng(1).random((60, 60)) < 0.3,
                                 np.random.default_rng(2).lognormal(0, 1, (60, 60)), 0.0))
    rp, col, val = (torch.as_tensor(x).cuda() for x in (er.row_ptr, er.col, er.val))
    v = torch.as_tensor(W.uniform_vector(3000, 1)).cuda()
    ent = torch.tensor([0, 17, 2999], dtype=torch.int32, device="cuda")
    counts = {}
    counts["plan_create"] = _oom_sweep(mcx, lambda: mcx.Plan(rp, col, val), _close)
    counts["plan_create_weighted_host"] = _oom_sweep(mcx, lambda: mcx.Plan.from_csr(wt), _close)

    def fresh(fn):
        def call():
            plan = mcx.Plan(rp, col, val)
            try:
                fn(plan)
            finally:
                plan.close()
        return call

    # first multi-chunk estimate of a plan grows its scratch; forward and TC grow theirs
    counts["estimate"] = _oom_sweep(mcx, fresh(lambda p: p.estimate(v, 0.1, 70000, entries=ent)))
    counts["forward"] = _oom_sweep(mcx, fresh(lambda p: p.forward(v, 0.1, 100000)))
    counts["total_communicability"] = _oom_sweep(mcx, fresh(lambda p: p.total_communicability(0.1, 100000)))
    counts["rqmc"] = _oom_sweep(mcx, fresh(lambda p: p.estimate_rqmc(v, 0.1, 6, 4, entries=ent)))
    counts["level_difference"] = _oom_sweep(mcx, fresh(lambda p: p.estimate_level_difference(v, 0.1, 8, 3000,
                                                                                            entries=ent)))
    h = [torch.as_tensor(x) for x in (er.row_ptr, er.col, er.val)] + [v.cpu()]
    counts["expm_multiply"] = _oom_sweep(mcx, lambda: mcx.expm_multiply(*h, t=None, paths=100))
    counts["mlp_create"] = _oom_sweep(mcx, lambda: mcx.MLP(seed=1), _close)
    X = torch.randn(3000, 5, device="cuda")
    y = torch.randn(3000, device="cuda")

    def fit():
        net = mcx.MLP(seed=1)
        try:
            net.fit(X, y, epochs=1, batch=512, lr=1e-3, seed=1)
        finally:
            net.close()
    counts["mlp_fit"] = _oom_sweep(mcx, fit)
    probs = [dict(row_ptr=er.row_ptr, col=er.col, val=er.val, v=W.uniform_vector(3000, 3), times=[0.1, 1.0],
                  paths=20000)]
    cache = str(tmp_path / "tune.jsonl")  # the warm call tunes, the failing ones read the cache
    counts["batch_create"] = _oom_sweep(mcx, lambda: mcx.Batch(probs, tune_cache=cache), _close)
    cprobs = [dict(row_ptr=er.row_ptr, col=er.col, val=er.val, v=W.uniform_vector(3000, 3), t=0.1, paths=100)]
    counts["cvbatch_create"] = _oom_sweep(mcx, lambda: mcx.CVBatch(cprobs, control="taylor", tune_cache=cache),
                                          _close)
    # every entry point made at least one allocation, so each was failed at least once
    assert all(c >= 1 for c in counts.values()), counts


def test_tensor_core_wait_gives_up_and_context_survives(mcx):
    from paper_1904_12759_gb300 import MCXError, _lib

    X = np.random.default_rng(0).normal(size=(1000, 5)).astype(np.float32)
    net = mcx.MLP(seed=5)
    prm = CV.init_params(9)
    net.set(np.concatenate([prm[k].ravel() for k in ("W1", "b1", "W2", "b2", "W3", "b3")]), np.zeros(5), np.ones(5))
    L = _lib.load()
    assert L.mcx_debug_mlp_wait_polls(net._h, 0) == 0
    net.predict(torch.as_tensor(X).cuda())
    with pytest.raises(MCXError) as ei:
        net.sync()
    assert ei.value.code == -7  # MCX_E_TIMEOUT
    assert L.mcx_debug_mlp_wait_polls(net._h, 0xFFFFFFFF) == 0
    y = net.predict(torch.as_tensor(X).cuda()).cpu().numpy()
    net.sync()
    X64 = X.astype(np.float64)
    oy, _ = CV.forward(prm, X64)
    assert np.all(np.abs(y - oy) <= CV.forward_error_bound(prm, X64))
    # the tensor-core gradient's waits: the same limit, the same latch
    t = np.random.default_rng(1).normal(size=1000).astype(np.float32)
    Xd, td = torch.as_tensor(X).cuda(), torch.as_tensor(t).cuda()
    assert L.mcx_debug_mlp_wait_polls(net._h, 0) == 0
    net.gradient(Xd, td)
    with pytest.raises(MCXError) as ei:
        net.sync()
    assert ei.value.code == -7
    assert L.mcx_debug_mlp_wait_polls(net._h, 0xFFFFFFFF) == 0
    g, _ = net.gradient(Xd, td)
    net.sync()
    _, og = CV.loss_and_grad(prm, X64, t.astype(np.float64))
    gb, _ = CV.gradient_error_bound(prm, X64, t.astype(np.float64))
    order = ("W1", "b1", "W2", "b2", "W3", "b3")
    assert np.all(np.abs(g.cpu().numpy() - np.concatenate([og[k].ravel() for k in order]))
                  <= np.concatenate([gb[k].ravel() for k in order]))
    net.close()
