"""Python front end of the mcx library: argument marshalling only.

Every step of the computation runs in the CUDA kernels behind the C-ABI;
this module turns torch tensors into device pointers and the current torch
stream into the stream argument.  PyTorch supplies device memory and streams.
"""
from __future__ import annotations

import ctypes as C

import torch

from . import _lib
from ._lib import FUNCTIONALS, PRECISIONS, check


def _stream(stream=None) -> C.c_void_p:
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


def _dev(t: torch.Tensor, dtype: torch.dtype, name: str) -> int:
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t.data_ptr()


def _host(t: torch.Tensor, dtype: torch.dtype, name: str) -> int:
    if t.dtype != dtype or t.is_cuda or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous host tensor of {dtype}")
    return t.data_ptr()


class Plan:
    """A prepared matrix A (Sec. 2: A = D - L) on the current CUDA device.

    ``Plan(row_ptr, col, val)`` with int64 / int32 / float64 tensors in CSR
    form, all on the GPU, or all on the host (they are then copied by the
    library inside the call).
    """

    def __init__(self, row_ptr: torch.Tensor, col: torch.Tensor, val: torch.Tensor, stream=None):
        L = _lib.load()
        n = row_ptr.numel() - 1
        nnz = col.numel()
        host = not row_ptr.is_cuda
        conv = _host if host else _dev
        p_rp = conv(row_ptr, torch.int64, "row_ptr")
        p_col = conv(col, torch.int32, "col") if nnz else 0
        p_val = conv(val, torch.float64, "val") if nnz else 0
        out = C.c_void_p()
        check(L.mcx_plan_create(n, nnz, C.c_void_p(p_rp), C.c_void_p(p_col), C.c_void_p(p_val),
                                _lib.PLAN_HOST_INPUT if host else 0, _stream(stream), C.byref(out)),
              "mcx_plan_create")
        self._h = out
        self.n = n
        self.nnz = nnz

    @classmethod
    def from_csr(cls, csr, device="cuda", stream=None) -> "Plan":
        """Build from any object with numpy row_ptr / col / val (e.g. workloads.CSR)."""
        rp = torch.as_tensor(csr.row_ptr, dtype=torch.int64)
        col = torch.as_tensor(csr.col, dtype=torch.int32)
        val = torch.as_tensor(csr.val, dtype=torch.float64)
        if device is not None and device != "cpu":
            rp, col, val = rp.to(device), col.to(device), val.to(device)
        return cls(rp, col, val, stream=stream)

    def info(self) -> dict:
        inf = _lib.PlanInfo()
        check(_lib.load().mcx_plan_get_info(self._h, C.byref(inf)), "mcx_plan_get_info")
        return {k: getattr(inf, k) for k, _ in inf._fields_ if k != "reserved"}

    def estimate(self, v: torch.Tensor, t: float, paths: int, entries: torch.Tensor | None = None, seed: int = 0,
                 path_offset: int = 0, mode: str = "exact", nsteps: int = 1, prec: str = "fp32",
                 out: tuple | None = None, stream=None):
        """Backward estimate of (exp(tA)v)_i for each entry (Theorem 1, Algorithm 1).

        Returns (mean, sem) float64 CUDA tensors of length len(entries) (or n).
        """
        L = _lib.load()
        p_v = _dev(v, torch.float64, "v")
        if v.numel() != self.n:
            raise ValueError("v must have n entries")
        if entries is None:
            ne, p_e = self.n, 0
        else:
            ne, p_e = entries.numel(), _dev(entries, torch.int32, "entries")
        if out is None:
            mean = torch.empty(ne, dtype=torch.float64, device=v.device)
            sem = torch.empty(ne, dtype=torch.float64, device=v.device)
        else:
            mean, sem = out
        p_sem = _dev(sem, torch.float64, "sem") if sem is not None else 0
        check(L.mcx_estimate(self._h, C.c_void_p(p_v), float(t), FUNCTIONALS[mode], int(nsteps), int(paths),
                             C.c_void_p(p_e), int(ne), int(seed), int(path_offset), PRECISIONS[prec],
                             C.c_void_p(_dev(mean, torch.float64, "mean")), C.c_void_p(p_sem), _stream(stream)),
              "mcx_estimate")
        return mean, sem

    def estimate_level_difference(self, v: torch.Tensor, t: float, nsteps: int, paths: int,
                                  entries: torch.Tensor | None = None, seed: int = 0, path_offset: int = 0,
                                  mode: str = "strang", prec: str = "fp32", out: tuple | None = None, stream=None):
        """Multilevel level difference: per entry the mean and standard error of
        v_{X_t} (W_N - W_{N/2}) over the paths of `estimate` with the same seed and
        offset (N = nsteps, even; STRANG or LIE).  Returns (mean, sem)."""
        L = _lib.load()
        p_v = _dev(v, torch.float64, "v")
        if v.numel() != self.n:
            raise ValueError("v must have n entries")
        if entries is None:
            ne, p_e = self.n, 0
        else:
            ne, p_e = entries.numel(), _dev(entries, torch.int32, "entries")
        if out is None:
            mean = torch.empty(ne, dtype=torch.float64, device=v.device)
            sem = torch.empty(ne, dtype=torch.float64, device=v.device)
        else:
            mean, sem = out
        p_sem = _dev(sem, torch.float64, "sem") if sem is not None else 0
        check(L.mcx_estimate_level_difference(self._h, C.c_void_p(p_v), float(t), FUNCTIONALS[mode], int(nsteps),
                                              int(paths), C.c_void_p(p_e), int(ne), int(seed), int(path_offset),
                                              PRECISIONS[prec], C.c_void_p(_dev(mean, torch.float64, "mean")),
                                              C.c_void_p(p_sem), _stream(stream)), "mcx_estimate_level_difference")
        return mean, sem

    def combine_levels(self, means, sems, stream=None):
        """Multilevel telescoping sum (mcx_combine_levels): per entry the sum of the
        level means and the root sum of squares of their standard errors."""
        L = len(means)
        n = means[0].numel()
        if len(sems) != L or any(m.numel() != n or s.numel() != n for m, s in zip(means, sems)):
            raise ValueError("one (mean, sem) pair of equal length per level")
        pm = (C.c_void_p * L)(*[_dev(m, torch.float64, "mean") for m in means])
        ps = (C.c_void_p * L)(*[_dev(s, torch.float64, "sem") for s in sems])
        mean = torch.empty(n, dtype=torch.float64, device=means[0].device)
        sem = torch.empty(n, dtype=torch.float64, device=means[0].device)
        check(_lib.load().mcx_combine_levels(L, n, pm, ps, C.c_void_p(mean.data_ptr()), C.c_void_p(sem.data_ptr()),
                                             _stream(stream)), "mcx_combine_levels")
        return mean, sem

    def estimate_rqmc(self, v: torch.Tensor, t: float, log2_points: int, replicates: int,
                      entries: torch.Tensor | None = None, seed: int = 0, mode: str = "exact", nsteps: int = 1,
                      prec: str = "fp32", replicate_offset: int = 0, out: tuple | None = None, stream=None):
        """Randomised quasi-Monte Carlo estimate of (exp(tA)v)_i: `replicates` scrambled
        Sobol' sets of 2^log2_points points (replicates replicate_offset ..; disjoint
        ranges merge with shard.merge) drive the first events of the paths.

        Returns (mean, sem) float64 CUDA tensors; sem comes from the spread of the
        replicate means.
        """
        L = _lib.load()
        p_v = _dev(v, torch.float64, "v")
        if v.numel() != self.n:
            raise ValueError("v must have n entries")
        if entries is None:
            ne, p_e = self.n, 0
        else:
            ne, p_e = entries.numel(), _dev(entries, torch.int32, "entries")
        if out is None:
            mean = torch.empty(ne, dtype=torch.float64, device=v.device)
            sem = torch.empty(ne, dtype=torch.float64, device=v.device)
        else:
            mean, sem = out
        p_sem = _dev(sem, torch.float64, "sem") if sem is not None else 0
        check(L.mcx_estimate_rqmc(self._h, C.c_void_p(p_v), float(t), FUNCTIONALS[mode], int(nsteps),
                                  int(log2_points), int(replicates), int(replicate_offset), C.c_void_p(p_e),
                                  int(ne), int(seed),
                                  PRECISIONS[prec], C.c_void_p(_dev(mean, torch.float64, "mean")),
                                  C.c_void_p(p_sem), _stream(stream)), "mcx_estimate_rqmc")
        return mean, sem

    def trace(self, t: float, entry: int, seed: int, first_path: int, count: int, mode: str = "exact",
              nsteps: int = 1, prec: str = "fp32", device="cuda", stream=None) -> dict:
        """Per-path end index, jump count, index hash and log-weight (for parity checks)."""
        L = _lib.load()
        out = {
            "end": torch.empty(count, dtype=torch.int32, device=device),
            "njumps": torch.empty(count, dtype=torch.int32, device=device),  # uint32 on the C side
            "hash": torch.empty(count, dtype=torch.int64, device=device),  # uint64 on the C side
            "logw": torch.empty(count, dtype=torch.float64, device=device),
        }
        check(L.mcx_trace_paths(self._h, float(t), FUNCTIONALS[mode], int(nsteps), int(entry), int(seed),
                                int(first_path), int(count), PRECISIONS[prec],
                                *[C.c_void_p(out[k].data_ptr()) for k in ("end", "njumps", "hash", "logw")],
                                _stream(stream)), "mcx_trace_paths")
        return out

    def forward(self, v: torch.Tensor, t: float, paths: int, seed: int = 0, path_offset: int = 0,
                mode: str = "exact", nsteps: int = 1, prec: str = "fp32", out: tuple | None = None, stream=None):
        """Forward full-vector estimate (Theorem 2, Algorithm 2); this plan must be built from A^T.

        Returns (x, sem) float64 CUDA tensors of length n."""
        p_v = _dev(v, torch.float64, "v")
        if v.numel() != self.n:
            raise ValueError("v must have n entries")
        if out is None:
            x = torch.empty(self.n, dtype=torch.float64, device=v.device)
            sem = torch.empty(self.n, dtype=torch.float64, device=v.device)
        else:
            x, sem = out
        p_sem = _dev(sem, torch.float64, "sem") if sem is not None else 0
        check(_lib.load().mcx_estimate_forward(self._h, C.c_void_p(p_v), float(t), FUNCTIONALS[mode], int(nsteps),
                                               int(paths), int(seed), int(path_offset), PRECISIONS[prec],
                                               C.c_void_p(_dev(x, torch.float64, "x")), C.c_void_p(p_sem),
                                               _stream(stream)), "mcx_estimate_forward")
        return x, sem

    def total_communicability(self, t: float, paths: int, mode: str = "exact", nsteps: int = 1, seed: int = 0,
                              path_offset: int = 0, prec: str = "fp32", out: tuple | None = None, stream=None):
        """TC(t) = 1^T exp(tA) 1 from the forward paths of v = 1 (plan of A^T); returns
        (tc, sem) as one-element device tensors."""
        dev = torch.device("cuda", torch.cuda.current_device())
        if out is None:
            tc = torch.empty(1, dtype=torch.float64, device=dev)
            sem = torch.empty(1, dtype=torch.float64, device=dev)
        else:
            tc, sem = out
        check(_lib.load().mcx_total_communicability(self._h, float(t), FUNCTIONALS[mode], int(nsteps), int(paths),
                                                    int(seed), int(path_offset), PRECISIONS[prec],
                                                    C.c_void_p(tc.data_ptr()), C.c_void_p(sem.data_ptr()),
                                                    _stream(stream)), "mcx_total_communicability")
        return tc, sem

    def trace_forward(self, v: torch.Tensor, t: float, seed: int, first_path: int, count: int, mode: str = "exact",
                      nsteps: int = 1, prec: str = "fp32", stream=None) -> dict:
        dev = v.device
        out = {
            "start": torch.empty(count, dtype=torch.int32, device=dev),
            "end": torch.empty(count, dtype=torch.int32, device=dev),
            "njumps": torch.empty(count, dtype=torch.int32, device=dev),
            "hash": torch.empty(count, dtype=torch.int64, device=dev),
            "logw": torch.empty(count, dtype=torch.float64, device=dev),
        }
        check(_lib.load().mcx_trace_forward(self._h, C.c_void_p(_dev(v, torch.float64, "v")), float(t),
                                            FUNCTIONALS[mode], int(nsteps), int(seed), int(first_path), int(count),
                                            PRECISIONS[prec],
                                            *[C.c_void_p(out[k].data_ptr()) for k in ("start", "end", "njumps",
                                                                                      "hash", "logw")],
                                            _stream(stream)), "mcx_trace_forward")
        return out

    def estimate_cv(self, coef: torch.Tensor, t: float, paths: int, entries: torch.Tensor | None = None,
                    seed: int = 0, path_offset: int = 0, prec: str = "fp32", out: tuple | None = None, stream=None):
        """Control-variate backward estimate (see cv_coefficients); returns (mean, sem)."""
        if entries is None:
            ne, p_e = self.n, 0
        else:
            ne, p_e = entries.numel(), _dev(entries, torch.int32, "entries")
        if out is None:
            mean = torch.empty(ne, dtype=torch.float64, device=coef.device)
            sem = torch.empty(ne, dtype=torch.float64, device=coef.device)
        else:
            mean, sem = out
        check(_lib.load().mcx_estimate_cv(self._h, C.c_void_p(_dev(coef, torch.float64, "coef")), float(t), int(paths),
                                          C.c_void_p(p_e), int(ne), int(seed), int(path_offset), PRECISIONS[prec],
                                          C.c_void_p(_dev(mean, torch.float64, "mean")),
                                          C.c_void_p(_dev(sem, torch.float64, "sem")), _stream(stream)),
              "mcx_estimate_cv")
        return mean, sem

    def export(self, stream=None) -> dict:
        """Copy the plan's preparation results (rates, potentials, jump tables) to new CUDA tensors."""
        inf = self.info()
        n, m = self.n, max(inf["nnz_off"], 1)
        dev = torch.device("cuda", torch.cuda.current_device())
        out = {
            "deg": torch.empty(n, dtype=torch.int32, device=dev),
            "row_start": torch.empty(n, dtype=torch.int64, device=dev),
            "weighted": torch.empty(n, dtype=torch.uint8, device=dev),
            "inv_rate32": torch.empty(n, dtype=torch.float32, device=dev),
            "delta32": torch.empty(n, dtype=torch.float32, device=dev),
            "inv_rate64": torch.empty(n, dtype=torch.float64, device=dev),
            "delta64": torch.empty(n, dtype=torch.float64, device=dev),
            "edge_col": torch.empty(m, dtype=torch.int32, device=dev),
            "alias_col": torch.empty(m, dtype=torch.int32, device=dev),
            "thresh": torch.empty(m, dtype=torch.int32, device=dev),  # uint32 on the C side
        }
        keys = ("deg", "row_start", "weighted", "inv_rate32", "delta32", "inv_rate64", "delta64", "edge_col",
                "alias_col", "thresh")
        check(_lib.load().mcx_plan_export(self._h, *[C.c_void_p(out[k].data_ptr()) for k in keys], _stream(stream)),
              "mcx_plan_export")
        return out

    def sync(self, stream=None) -> dict:
        st = _lib.Stats()
        check(_lib.load().mcx_sync(self._h, _stream(stream), C.byref(st)), "mcx_sync")
        return {"paths": st.paths, "jumps": st.jumps, "status_bits": st.status_bits}

    def close(self) -> None:
        if getattr(self, "_h", None):
            _lib.load().mcx_plan_destroy(self._h)
            self._h = None

    def __del__(self):  # pragma: no cover - interpreter shutdown ordering
        try:
            self.close()
        except Exception:
            pass


def gather_rate(buffer_bytes: int, dependent: bool = True, loads: int = 1 << 31, stream=None) -> float:
    """Random 32-byte-sector gathers per second from a device buffer of `buffer_bytes`
    (dependent chains as in the walkers, or independent loads): the measured
    gather roofline, from L2 for a buffer that fits in it, from HBM otherwise."""
    out = C.c_double(0.0)
    check(_lib.load().mcx_gather_rate(int(buffer_bytes), 1 if dependent else 0, int(loads), C.byref(out),
                                      _stream(stream)), "mcx_gather_rate")
    return out.value


def power_iteration(row_ptr: torch.Tensor, col: torch.Tensor, val: torch.Tensor, max_iters: int = 1000,
                    tol: float = 1e-12, work: torch.Tensor | None = None, stream=None):
    """lambda_max of a symmetric A >= 0 by the power method on the GPU (Sec. 6: beta = 1/lambda_max).

    Returns (lambda, iterations)."""
    n = row_ptr.numel() - 1
    if work is None:
        work = torch.empty(3 * n + 4096, dtype=torch.float64, device=row_ptr.device)
    lam = C.c_double()
    it = C.c_int32()
    check(_lib.load().mcx_power_iteration(n, C.c_void_p(_dev(row_ptr, torch.int64, "row_ptr")),
                                          C.c_void_p(_dev(col, torch.int32, "col")),
                                          C.c_void_p(_dev(val, torch.float64, "val")), int(max_iters), float(tol),
                                          C.c_void_p(_dev(work, torch.float64, "work")), C.byref(lam), C.byref(it),
                                          _stream(stream)), "mcx_power_iteration")
    return lam.value, it.value


def expm_multiply(row_ptr: torch.Tensor, col: torch.Tensor, val: torch.Tensor, v: torch.Tensor,
                  t: float | None = None, beta_scale: float = 1.0, paths: int = 1000,
                  entries: torch.Tensor | None = None, seed: int = 0, path_offset: int = 0, mode: str = "exact",
                  nsteps: int = 1, prec: str = "fp32", out: tuple | None = None, stream=None):
    """x ~ exp(tA) v in one call of mcx_expm_multiply: plan, optional beta setup,
    backward estimate, status check.

    With t=None the horizon is beta_scale / lambda_max(A) (Sec. 6 uses
    beta = 1/lambda_max), lambda_max by the GPU power method.  All tensors on
    the host (page-locked for asynchronous copies): the library copies the
    inputs to the current device and the results back inside the call; all on
    the device: they are used in place.  Returns (mean, sem, t).
    """
    host = not row_ptr.is_cuda
    tensors = [row_ptr, col, val, v] + ([entries] if entries is not None else [])
    if any(x.is_cuda == host for x in tensors):
        raise ValueError("expm_multiply: the arrays must be all on the host or all on the device")
    n = row_ptr.numel() - 1
    ne = n if entries is None else entries.numel()
    if out is None:
        kw = dict(dtype=torch.float64, pin_memory=host and torch.cuda.is_available()) if host else \
            dict(dtype=torch.float64, device=v.device)
        mean, sem = torch.empty(ne, **kw), torch.empty(ne, **kw)
    else:
        mean, sem = out

    def ptr(x, dt, name):
        if x.dtype != dt or not x.is_contiguous():
            raise ValueError(f"{name} must be a contiguous {dt} tensor")
        return C.c_void_p(x.data_ptr())

    t_used = C.c_double(0.0)
    check(_lib.load().mcx_expm_multiply(
        n, col.numel(), ptr(row_ptr, torch.int64, "row_ptr"), ptr(col, torch.int32, "col"),
        ptr(val, torch.float64, "val"), ptr(v, torch.float64, "v"), -1.0 if t is None else float(t),
        float(beta_scale), FUNCTIONALS[mode], int(nsteps), int(paths),
        ptr(entries, torch.int32, "entries") if entries is not None else C.c_void_p(0), int(ne), int(seed),
        int(path_offset), PRECISIONS[prec], _lib.PLAN_HOST_INPUT if host else 0, ptr(mean, torch.float64, "mean"),
        ptr(sem, torch.float64, "sem") if sem is not None else C.c_void_p(0), C.byref(t_used), _stream(stream)),
        "mcx_expm_multiply")
    return mean, sem, t_used.value


class Batch:
    """Many forward problems (Theorem 2) in one persistent, graph-captured launch.

    ``problems``: list of dicts with numpy/torch host arrays ``row_ptr``, ``col``,
    ``val`` (the plan matrix B = A^T), ``v`` (>= 0), ``times`` and ``paths``
    (forward paths per time).  ``tune_cache``: path of the schedule cache file.
    """

    def __init__(self, problems, tune_cache: str | None = None, stream=None):
        import numpy as np

        L = _lib.load()
        self._keep = []
        arr = (_lib.Problem * len(problems))()
        self.sizes = []
        for k, p in enumerate(problems):
            rp = np.ascontiguousarray(p["row_ptr"], dtype=np.int64)
            col = np.ascontiguousarray(p["col"], dtype=np.int32)
            val = np.ascontiguousarray(p["val"], dtype=np.float64)
            v = np.ascontiguousarray(p["v"], dtype=np.float64)
            times = np.ascontiguousarray(p["times"], dtype=np.float64)
            self._keep += [rp, col, val, v, times]
            arr[k] = _lib.Problem(rp.size - 1, col.size, rp.ctypes.data, col.ctypes.data, val.ctypes.data,
                                  v.ctypes.data, times.size, times.ctypes.data, int(p["paths"]))
            self.sizes.append((rp.size - 1, times.size))
        out = C.c_void_p()
        check(L.mcx_batch_create(len(problems), arr, tune_cache.encode() if tune_cache else None,
                                 _stream(stream), C.byref(out)), "mcx_batch_create")
        self._keep = None
        self._h = out

    def info(self) -> dict:
        inf = _lib.BatchInfo()
        check(_lib.load().mcx_batch_get_info(self._h, C.byref(inf)), "mcx_batch_get_info")
        return {k: getattr(inf, k) for k, _ in inf._fields_ if k != "reserved"}

    def run(self, seed: int, stream=None) -> None:
        check(_lib.load().mcx_batch_run(self._h, int(seed), _stream(stream)), "mcx_batch_run")

    def set_v(self, problem: int, v, stream=None) -> None:
        """New start vector of one problem for the next runs (tables rebuilt in the graph)."""
        n = self.sizes[problem][0]
        if v.numel() != n:
            raise ValueError("v must have the problem's n entries")
        check(_lib.load().mcx_batch_set_v(self._h, int(problem), C.c_void_p(_dev(v, torch.float64, "v")),
                                          _stream(stream)), "mcx_batch_set_v")

    def result(self, problem: int, time_index: int, stream=None):
        n = self.sizes[problem][0]
        dev = torch.device("cuda", torch.cuda.current_device())
        x = torch.empty(n, dtype=torch.float64, device=dev)
        sem = torch.empty(n, dtype=torch.float64, device=dev)
        check(_lib.load().mcx_batch_result(self._h, int(problem), int(time_index), C.c_void_p(x.data_ptr()),
                                           C.c_void_p(sem.data_ptr()), _stream(stream)), "mcx_batch_result")
        return x, sem

    def sync(self, stream=None) -> dict:
        st = _lib.Stats()
        check(_lib.load().mcx_batch_sync(self._h, _stream(stream), C.byref(st)), "mcx_batch_sync")
        return {"paths": st.paths, "jumps": st.jumps, "status_bits": st.status_bits}

    def close(self) -> None:
        if getattr(self, "_h", None):
            _lib.load().mcx_batch_destroy(self._h)
            self._h = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# Learned control variate
# ---------------------------------------------------------------------------
def cv_prepare(row_ptr, col, val, v, t: float, stream=None):
    """Taylor terms [4, n] (v, Av, A^2v, A^3v) and node features [n, 5] of (A, v, t)."""
    n = row_ptr.numel() - 1
    dev = row_ptr.device
    work = torch.empty(3 * n + 64, dtype=torch.float64, device=dev)
    taylor = torch.empty(4 * n, dtype=torch.float64, device=dev)
    feat = torch.empty(5 * n, dtype=torch.float32, device=dev)
    check(_lib.load().mcx_cv_prepare(n, C.c_void_p(_dev(row_ptr, torch.int64, "row_ptr")),
                                     C.c_void_p(_dev(col, torch.int32, "col")),
                                     C.c_void_p(_dev(val, torch.float64, "val")),
                                     C.c_void_p(_dev(v, torch.float64, "v")), float(t), C.c_void_p(work.data_ptr()),
                                     C.c_void_p(taylor.data_ptr()), C.c_void_p(feat.data_ptr()), _stream(stream)),
          "mcx_cv_prepare")
    return taylor.view(4, n), feat.view(n, 5)


def cv_targets(x, taylor, t: float, stream=None):
    n = x.numel()
    y = torch.empty(n, dtype=torch.float32, device=x.device)
    check(_lib.load().mcx_cv_targets(n, C.c_void_p(_dev(x, torch.float64, "x")),
                                     C.c_void_p(_dev(taylor.contiguous(), torch.float64, "taylor")), float(t),
                                     C.c_void_p(y.data_ptr()), _stream(stream)), "mcx_cv_targets")
    return y


def cv_coefficients(row_ptr, col, val, taylor, y, t: float, stream=None):
    """coef [3n] = [(a, b) pairs | xhat] for mcx_estimate_cv (y None: Taylor-only)."""
    n = row_ptr.numel() - 1
    dev = row_ptr.device
    work = torch.empty(3 * n + 64, dtype=torch.float64, device=dev)
    coef = torch.empty(3 * n, dtype=torch.float64, device=dev)
    p_y = _dev(y, torch.float32, "y") if y is not None else 0
    check(_lib.load().mcx_cv_coefficients(n, C.c_void_p(_dev(row_ptr, torch.int64, "row_ptr")),
                                          C.c_void_p(_dev(col, torch.int32, "col")),
                                          C.c_void_p(_dev(val, torch.float64, "val")),
                                          C.c_void_p(_dev(taylor.contiguous(), torch.float64, "taylor")),
                                          C.c_void_p(p_y), float(t), C.c_void_p(work.data_ptr()),
                                          C.c_void_p(coef.data_ptr()), _stream(stream)), "mcx_cv_coefficients")
    return coef


class MLP:
    """The 5-64-64-1 control-variate network (BF16 weights in use, FP32 master;
    inference on the tensor cores with the first hidden layer rounded to BF16)."""

    NPARAM = 4609

    def __init__(self, seed: int = 0):
        out = C.c_void_p()
        check(_lib.load().mcx_mlp_create(int(seed), C.byref(out)), "mcx_mlp_create")
        self._h = out

    def get(self):
        import numpy as np

        p = np.zeros(self.NPARAM, np.float32)
        mu = np.zeros(5, np.float32)
        sd = np.zeros(5, np.float32)
        check(_lib.load().mcx_mlp_get(self._h, p.ctypes.data, mu.ctypes.data, sd.ctypes.data), "mcx_mlp_get")
        return p, mu, sd

    def set(self, params=None, mu=None, sd=None):
        import numpy as np

        arrs = [None if a is None else np.ascontiguousarray(a, dtype=np.float32) for a in (params, mu, sd)]
        check(_lib.load().mcx_mlp_set(self._h, *[None if a is None else a.ctypes.data for a in arrs]),
              "mcx_mlp_set")

    def predict(self, features, stream=None):
        n = features.shape[0]
        y = torch.empty(n, dtype=torch.float32, device=features.device)
        check(_lib.load().mcx_mlp_predict(self._h, n, C.c_void_p(_dev(features.contiguous(), torch.float32, "f")),
                                          C.c_void_p(y.data_ptr()), _stream(stream)), "mcx_mlp_predict")
        return y

    def sync(self, stream=None):
        """Synchronise and raise if an inference call latched a device error."""
        check(_lib.load().mcx_mlp_sync(self._h, _stream(stream)), "mcx_mlp_sync")

    def gradient(self, features, targets, stream=None):
        g = torch.empty(self.NPARAM, dtype=torch.float32, device=features.device)
        loss = C.c_float()
        check(_lib.load().mcx_mlp_gradient(self._h, features.shape[0],
                                           C.c_void_p(_dev(features.contiguous(), torch.float32, "f")),
                                           C.c_void_p(_dev(targets, torch.float32, "targets")),
                                           C.c_void_p(g.data_ptr()), C.byref(loss), _stream(stream)),
              "mcx_mlp_gradient")
        return g, loss.value

    def fit(self, features, targets, epochs=20, batch=4096, lr=1e-3, seed=0, stream=None):
        import numpy as np

        losses = np.zeros(max(epochs, 1), np.float32)
        check(_lib.load().mcx_mlp_fit(self._h, features.shape[0],
                                      C.c_void_p(_dev(features.contiguous(), torch.float32, "f")),
                                      C.c_void_p(_dev(targets, torch.float32, "targets")), int(epochs), int(batch),
                                      float(lr), int(seed), losses.ctypes.data, _stream(stream)), "mcx_mlp_fit")
        return losses[:epochs]

    def close(self):
        if getattr(self, "_h", None):
            _lib.load().mcx_mlp_destroy(self._h)
            self._h = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass


class CVBatch:
    """Many backward full-vector estimates (Theorem 1) with the control variate of
    Sec. 5 in one CUDA-graph launch per run (mcx_cvbatch_*).

    ``problems``: list of dicts with host arrays ``row_ptr``, ``col``, ``val`` (the CSR
    of A), ``v`` (n values, or n_rhs x n for several right-hand sides), ``t`` (a scalar
    or one horizon per right-hand side) and ``paths`` (paths per entry).
    ``control``: "none" (plain estimate), "taylor" or "learned" (needs ``net``, an
    :class:`MLP`).  ``prec``: "fp32" or "fp64" (plain: the FP64 path version; control
    variates: residual integrals in FP64).  Pair k (problems in order, right-hand
    sides in order) simulates paths k * 2^40 + p of each entry.
    """

    def __init__(self, problems, control: str = "learned", net=None, prec: str = "fp32",
                 tune_cache: str | None = None, stream=None):
        import numpy as np

        L = _lib.load()
        keep = []
        arr = (_lib.CvProblem * len(problems))()
        self.sizes = []
        for k, p in enumerate(problems):
            rp = np.ascontiguousarray(p["row_ptr"], dtype=np.int64)
            col = np.ascontiguousarray(p["col"], dtype=np.int32)
            val = np.ascontiguousarray(p["val"], dtype=np.float64)
            n = rp.size - 1
            v = np.ascontiguousarray(np.asarray(p["v"], dtype=np.float64).reshape(-1, n))
            t = np.ascontiguousarray(np.broadcast_to(np.asarray(p["t"], dtype=np.float64), (v.shape[0],)))
            keep += [rp, col, val, v, t]
            arr[k] = _lib.CvProblem(n, col.size, rp.ctypes.data, col.ctypes.data, val.ctypes.data, v.shape[0],
                                    v.ctypes.data, t.ctypes.data, int(p["paths"]))
            self.sizes.append((n, v.shape[0]))
        out = C.c_void_p()
        self.control = control
        check(L.mcx_cvbatch_create(len(problems), arr, _lib.CV_CONTROLS[control],
                                   net._h if net is not None else None, PRECISIONS[prec],
                                   tune_cache.encode() if tune_cache else None, _stream(stream), C.byref(out)),
              "mcx_cvbatch_create")
        self._h = out

    def info(self) -> dict:
        inf = _lib.CvBatchInfo()
        check(_lib.load().mcx_cvbatch_get_info(self._h, C.byref(inf)), "mcx_cvbatch_get_info")
        return {k: getattr(inf, k) for k, _ in inf._fields_}

    def set_paths(self, paths, stream=None) -> None:
        import numpy as np

        p = np.ascontiguousarray(np.broadcast_to(np.asarray(paths, dtype=np.uint64), (len(self.sizes),)))
        check(_lib.load().mcx_cvbatch_set_paths(self._h, C.c_void_p(p.ctypes.data), _stream(stream)),
              "mcx_cvbatch_set_paths")

    def run(self, seed: int, stream=None) -> None:
        check(_lib.load().mcx_cvbatch_run(self._h, int(seed), _stream(stream)), "mcx_cvbatch_run")

    def result(self, problem: int, rhs: int = 0, stream=None):
        n = self.sizes[problem][0]
        dev = torch.device("cuda", torch.cuda.current_device())
        x = torch.empty(n, dtype=torch.float64, device=dev)
        sem = torch.empty(n, dtype=torch.float64, device=dev)
        check(_lib.load().mcx_cvbatch_result(self._h, int(problem), int(rhs), C.c_void_p(x.data_ptr()),
                                             C.c_void_p(sem.data_ptr()), _stream(stream)), "mcx_cvbatch_result")
        return x, sem

    def coefficients(self, problem: int, rhs: int = 0, stream=None):
        n = self.sizes[problem][0]
        coef = torch.empty(3 * n, dtype=torch.float64, device=torch.device("cuda", torch.cuda.current_device()))
        check(_lib.load().mcx_cvbatch_coefficients(self._h, int(problem), int(rhs), C.c_void_p(coef.data_ptr()),
                                                   _stream(stream)), "mcx_cvbatch_coefficients")
        return coef

    def sync(self, stream=None) -> dict:
        st = _lib.Stats()
        check(_lib.load().mcx_cvbatch_sync(self._h, _stream(stream), C.byref(st)), "mcx_cvbatch_sync")
        return {"paths": st.paths, "jumps": st.jumps, "status_bits": st.status_bits}

    def close(self) -> None:
        if getattr(self, "_h", None):
            _lib.load().mcx_cvbatch_destroy(self._h)
            self._h = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass


def debug_fail_alloc(k: int) -> int:
    """Test hook: the k-th device allocation of the library from now fails (k <= 0
    disarms); returns the library's allocation count so far."""
    return int(_lib.load().mcx_debug_fail_alloc(int(k)))


def debug_pool_usage() -> tuple:
    """(bytes in use, bytes reserved) of the library's memory pool on the current device."""
    u, r = C.c_uint64(0), C.c_uint64(0)
    check(_lib.load().mcx_debug_pool_usage(C.byref(u), C.byref(r)), "mcx_debug_pool_usage")
    return u.value, r.value
