"""ctypes front end of the C oracle walker (test infrastructure only).

``build()`` compiles walker.c with gcc (-O2 -ffp-contract=off -fno-fast-math,
OpenMP when available) into oracle/_build/.  The functions below mirror the
library's calls but run the plain sequential statement of the method in
walker.c: Sec. 3 (path sampler), Algorithms 1-2, Theorems 1-2.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "walker.c")
_OUT = os.path.join(_HERE, "_build", "liboracle_walker.so")
_lock = threading.Lock()
_lib = None

MODES = {"exact": 0, "strang": 1, "lie": 2}
START_GROUP = 1024  # group size of the two-level start table (walker.c)
PRECS = {"fp32": 0, "fp64": 1}


def build(force: bool = False) -> str:
    """Compile walker.c (only when the source is newer than the library)."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if not force and os.path.exists(_OUT) and os.path.getmtime(_OUT) >= os.path.getmtime(_SRC):
        return _OUT
    base = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC", _SRC, "-lm"]
    tmp = _OUT + f".tmp{os.getpid()}"
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:] + ["-o", tmp], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base + ["-o", tmp], check=True)
    os.replace(tmp, _OUT)
    return _OUT


class _Graph(C.Structure):
    _fields_ = [
        ("n", C.c_int64), ("nnz_off", C.c_int64),
        ("deg", C.c_void_p), ("row_start", C.c_void_p), ("weighted", C.c_void_p),
        ("inv_rate32", C.c_void_p), ("delta32", C.c_void_p),
        ("inv_rate64", C.c_void_p), ("delta64", C.c_void_p),
        ("edge_col", C.c_void_p), ("alias_col", C.c_void_p), ("thresh", C.c_void_p),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = C.CDLL(path)
            vp, i64, u64, i32, u32, dbl = C.c_void_p, C.c_int64, C.c_uint64, C.c_int32, C.c_uint32, C.c_double
            L.oracle_philox4x32_10.argtypes = [vp, vp, vp]
            L.oracle_logf.argtypes = [C.c_float]
            L.oracle_logf.restype = C.c_float
            L.oracle_logf_many.argtypes = [vp, vp, i64]
            L.oracle_ln_table.argtypes = [vp, vp]
            L.oracle_log.argtypes = [dbl]
            L.oracle_log.restype = dbl
            L.oracle_count_offdiag.argtypes = [i64, vp, vp, vp]
            L.oracle_count_offdiag.restype = i64
            L.oracle_prep.argtypes = [i64, vp, vp, vp, C.POINTER(_Graph)]
            L.oracle_prep.restype = C.c_int
            L.oracle_trace.argtypes = [C.POINTER(_Graph), dbl, C.c_int, C.c_int, C.c_int, i32, u64, u64, u32,
                                       vp, vp, vp, vp]
            L.oracle_estimate.argtypes = [C.POINTER(_Graph), vp, dbl, C.c_int, C.c_int, C.c_int, u64, vp, i64,
                                          u64, u64, vp, vp, vp]
            L.oracle_estimate.restype = C.c_int
            L.oracle_start_table.argtypes = [i64, vp, vp, vp, vp, vp, vp]
            L.oracle_start_table.restype = C.c_int
            L.oracle_forward.argtypes = [C.POINTER(_Graph), i64, vp, vp, vp, vp, dbl, dbl, C.c_int, C.c_int,
                                         C.c_int, u64, u64, u64, vp, vp, vp]
            L.oracle_forward_trace.argtypes = [C.POINTER(_Graph), i64, vp, vp, vp, vp, dbl, C.c_int, C.c_int,
                                               C.c_int, u64, u64, u32, vp, vp, vp, vp, vp]
            L.oracle_phi.argtypes = [C.c_int, dbl]
            L.oracle_phi.restype = dbl
            L.oracle_estimate_cv.argtypes = [C.POINTER(_Graph), vp, vp, vp, dbl, u64, vp, i64, u64, u64, vp, vp]
            L.oracle_estimate_cv.restype = C.c_int
            L.oracle_num_threads.restype = C.c_int
            L.oracle_qmc_dims.restype = C.c_int
            L.oracle_sobol_poly.argtypes = [C.c_int, vp, vp]
            L.oracle_sobol_directions.argtypes = [vp]
            L.oracle_sobol_point.argtypes = [vp, u32]
            L.oracle_sobol_point.restype = u32
            L.oracle_qmc_scrambled.argtypes = [u64, u32, vp]
            L.oracle_qmc_shift.argtypes = [u64, i32, u32, u32]
            L.oracle_qmc_shift.restype = u32
            L.oracle_estimate_rqmc.argtypes = [C.POINTER(_Graph), vp, dbl, C.c_int, C.c_int, C.c_int, u32, u32, u32,
                                               vp, i64, u64, vp, vp, vp, vp]
            L.oracle_estimate_rqmc.restype = C.c_int
            L.oracle_estimate_level_difference.argtypes = [C.POINTER(_Graph), vp, dbl, C.c_int, C.c_int, C.c_int,
                                                           u64, vp, i64, u64, u64, vp, vp]
            L.oracle_estimate_level_difference.restype = C.c_int
            L.oracle_trace_rqmc.argtypes = [C.POINTER(_Graph), dbl, C.c_int, C.c_int, C.c_int, i32, u64, u32, u32,
                                            u32, u32, vp, vp, vp, vp]
            _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().oracle_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def logf(x: float) -> float:
    return float(np.float32(lib().oracle_logf(float(x))))


def logf_many(x) -> np.ndarray:
    """The FP32 logarithm of every element of x (float32 array)."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    y = np.empty_like(x)
    lib().oracle_logf_many(_p(x), _p(y), int(x.size))
    return y


def ln_table():
    """The FP32 logarithm's breakpoint table: (1/c_j, L_j) for j = 0..64."""
    inv = np.empty(65, np.float32)
    L = np.empty(65, np.float32)
    lib().oracle_ln_table(_p(inv), _p(L))
    return inv, L


def log(x: float) -> float:
    return float(lib().oracle_log(float(x)))


class Graph:
    """The oracle's prepared form of A = D - L: rates, potentials and jump tables."""

    def __init__(self, csr):
        n = int(csr.n)
        self.n = n
        self.row_ptr = np.ascontiguousarray(csr.row_ptr, dtype=np.int64)
        self.col = np.ascontiguousarray(csr.col, dtype=np.int32)
        self.val = np.ascontiguousarray(csr.val, dtype=np.float64)
        L = lib()
        m = int(L.oracle_count_offdiag(n, _p(self.row_ptr), _p(self.col), _p(self.val)))
        self.deg = np.zeros(n, np.int32)
        self.row_start = np.zeros(n, np.int64)
        self.weighted = np.zeros(n, np.uint8)
        self.inv_rate32 = np.zeros(n, np.float32)
        self.delta32 = np.zeros(n, np.float32)
        self.inv_rate64 = np.zeros(n, np.float64)
        self.delta64 = np.zeros(n, np.float64)
        self.edge_col = np.zeros(max(m, 1), np.int32)
        self.alias_col = np.zeros(max(m, 1), np.int32)
        self.thresh = np.zeros(max(m, 1), np.uint32)
        self._g = _Graph(n, 0, *[a.ctypes.data for a in (
            self.deg, self.row_start, self.weighted, self.inv_rate32, self.delta32,
            self.inv_rate64, self.delta64, self.edge_col, self.alias_col, self.thresh)])
        self.status = int(L.oracle_prep(n, _p(self.row_ptr), _p(self.col), _p(self.val), C.byref(self._g)))
        self.nnz_off = int(self._g.nnz_off)

    def trace(self, t, entry, seed, first_path, count, mode="exact", nsteps=1, prec="fp32"):
        end = np.zeros(count, np.int32)
        nj = np.zeros(count, np.uint32)
        hs = np.zeros(count, np.uint64)
        lw = np.zeros(count, np.float64)
        lib().oracle_trace(C.byref(self._g), float(t), MODES[mode], int(nsteps), PRECS[prec], int(entry),
                           int(seed), int(first_path), int(count), _p(end), _p(nj), _p(hs), _p(lw))
        return {"end": end, "njumps": nj, "hash": hs, "logw": lw}

    def estimate(self, v, t, paths, entries=None, seed=0, path_offset=0, mode="exact", nsteps=1, prec="fp32"):
        """Per-entry sample mean of W v_{X_t} and its standard error (Algorithm 1)."""
        v = np.ascontiguousarray(v, dtype=np.float64)
        if entries is None:
            ne = self.n
            ent_p = None
        else:
            entries = np.ascontiguousarray(entries, dtype=np.int32)
            ne = entries.size
            ent_p = _p(entries)
        mean = np.zeros(ne)
        sem = np.zeros(ne)
        jumps = np.zeros(1, np.uint64)
        lib().oracle_estimate(C.byref(self._g), _p(v), float(t), MODES[mode], int(nsteps), PRECS[prec],
                              int(paths), ent_p, int(ne), int(seed), int(path_offset), _p(mean), _p(sem),
                              _p(jumps))
        return mean, sem, int(jumps[0])

    def estimate_cv(self, a, b, h, t, paths, entries=None, seed=0, path_offset=0):
        """Control-variate estimate h_i + mean residual integral (FP32 paths, EXACT)."""
        a = np.ascontiguousarray(a, dtype=np.float64)
        b = np.ascontiguousarray(b, dtype=np.float64)
        h = np.ascontiguousarray(h, dtype=np.float64)
        if entries is None:
            ne, ent_p = self.n, None
        else:
            entries = np.ascontiguousarray(entries, dtype=np.int32)
            ne, ent_p = entries.size, _p(entries)
        mean = np.zeros(ne)
        sem = np.zeros(ne)
        lib().oracle_estimate_cv(C.byref(self._g), _p(a), _p(b), _p(h), float(t), int(paths), ent_p, int(ne),
                                 int(seed), int(path_offset), _p(mean), _p(sem))
        return mean, sem

    def estimate_rqmc(self, v, t, log2q, replicates, entries=None, seed=0, mode="exact", nsteps=1, prec="fp32",
                      replicate_offset=0):
        """Randomised-QMC estimate: per entry, the mean of `replicates` replicate means (replicates
        replicate_offset ..) over the 2^log2q scrambled Sobol' points, its standard error from
        their spread, and the replicate means themselves [entries, replicates]."""
        v = np.ascontiguousarray(v, dtype=np.float64)
        if entries is None:
            ne, ent_p = self.n, None
        else:
            entries = np.ascontiguousarray(entries, dtype=np.int32)
            ne, ent_p = entries.size, _p(entries)
        mean = np.zeros(ne)
        sem = np.zeros(ne)
        reps = np.zeros((ne, int(replicates)))
        jumps = np.zeros(1, np.uint64)
        st = lib().oracle_estimate_rqmc(C.byref(self._g), _p(v), float(t), MODES[mode], int(nsteps), PRECS[prec],
                                        int(log2q), int(replicates), int(replicate_offset), ent_p, int(ne),
                                        int(seed), _p(mean), _p(sem), _p(reps), _p(jumps))
        if st != 0:
            raise ValueError("invalid quasi-random set size")
        return mean, sem, reps

    def estimate_level_difference(self, v, t, nsteps, paths, entries=None, seed=0, path_offset=0, mode="strang",
                                  prec="fp32"):
        """Multilevel difference: per entry the mean and standard error of
        v_{X_t} (W_N - W_{N/2}) over the same paths (N = nsteps, even)."""
        v = np.ascontiguousarray(v, dtype=np.float64)
        if entries is None:
            ne, ent_p = self.n, None
        else:
            entries = np.ascontiguousarray(entries, dtype=np.int32)
            ne, ent_p = entries.size, _p(entries)
        mean = np.zeros(ne)
        sem = np.zeros(ne)
        st = lib().oracle_estimate_level_difference(C.byref(self._g), _p(v), float(t), MODES[mode], int(nsteps),
                                                    PRECS[prec], int(paths), ent_p, int(ne), int(seed),
                                                    int(path_offset), _p(mean), _p(sem))
        if st != 0:
            raise ValueError("level differences need STRANG or LIE with an even step count")
        return mean, sem

    def trace_rqmc(self, t, entry, seed, log2q, replicate, first_point, count, mode="exact", nsteps=1, prec="fp32"):
        end = np.zeros(count, np.int32)
        nj = np.zeros(count, np.uint32)
        hs = np.zeros(count, np.uint64)
        lw = np.zeros(count, np.float64)
        lib().oracle_trace_rqmc(C.byref(self._g), float(t), MODES[mode], int(nsteps), PRECS[prec], int(entry),
                                int(seed), int(log2q), int(replicate), int(first_point), int(count), _p(end),
                                _p(nj), _p(hs), _p(lw))
        return {"end": end, "njumps": nj, "hash": hs, "logw": lw}

    # -- forward form (Theorem 2, Algorithm 2); this graph must be that of A^T --
    def start_table(self, v):
        """Two-level alias tables for the start draw j ~ v/V (Lemma 2)."""
        v = np.ascontiguousarray(v, dtype=np.float64)
        G = (self.n + START_GROUP - 1) // START_GROUP
        t = {"top_alias": np.zeros(max(G, 1), np.int32), "top_thresh": np.zeros(max(G, 1), np.uint32),
             "in_alias": np.zeros(self.n, np.int32), "in_thresh": np.zeros(self.n, np.uint32)}
        vs = np.zeros(1)
        st = int(lib().oracle_start_table(self.n, _p(v), _p(t["top_alias"]), _p(t["top_thresh"]),
                                          _p(t["in_alias"]), _p(t["in_thresh"]), _p(vs)))
        t["V"] = float(vs[0])
        return st, t

    def _tables(self, v):
        st, t = self.start_table(v)
        if st != 0:
            raise ValueError("forward form needs v >= 0 with a positive sum")
        return t, [_p(t[k]) for k in ("top_alias", "top_thresh", "in_alias", "in_thresh")]

    def forward(self, v, t, total_paths, seed=0, path_offset=0, mode="exact", nsteps=1, prec="fp32"):
        """Full-vector estimate x_i = V E[W 1{X_t=i}] with its standard error."""
        tab, ptrs = self._tables(v)
        s1 = np.zeros(self.n)
        s2 = np.zeros(self.n)
        jumps = np.zeros(1, np.uint64)
        lib().oracle_forward(C.byref(self._g), self.n, *ptrs, tab["V"], float(t), MODES[mode], int(nsteps),
                             PRECS[prec], int(total_paths), int(seed), int(path_offset), _p(s1), _p(s2),
                             _p(jumps))
        M = float(total_paths)
        x = s1 / M
        var = np.maximum(s2 / M - x * x, 0.0) * (M / max(M - 1.0, 1.0))
        return x, np.sqrt(var / M), int(jumps[0])

    def forward_trace(self, v, t, seed, first_path, count, mode="exact", nsteps=1, prec="fp32"):
        tab, ptrs = self._tables(v)
        out = {k: np.zeros(count, dt) for k, dt in (("start", np.int32), ("end", np.int32), ("njumps", np.uint32),
                                                    ("hash", np.uint64), ("logw", np.float64))}
        lib().oracle_forward_trace(C.byref(self._g), self.n, *ptrs, float(t), MODES[mode], int(nsteps),
                                   PRECS[prec], int(seed), int(first_path), int(count), _p(out["start"]),
                                   _p(out["end"]), _p(out["njumps"]), _p(out["hash"]), _p(out["logw"]))
        return out


def phi(k: int, z: float) -> float:
    """int_0^1 e^{zs} s^k ds (the oracle's evaluation)."""
    return float(lib().oracle_phi(int(k), float(z)))


def qmc_dims() -> int:
    return int(lib().oracle_qmc_dims())


def sobol_poly(d: int):
    """(degree, coefficient bits) of the primitive polynomial of Sobol' dimension d >= 1."""
    s = np.zeros(1, np.int32)
    a = np.zeros(1, np.int32)
    lib().oracle_sobol_poly(int(d), _p(s), _p(a))
    return int(s[0]), int(a[0])


def sobol_directions() -> np.ndarray:
    """Unscrambled direction numbers [dims, 32] (uint32)."""
    V = np.zeros((qmc_dims(), 32), np.uint32)
    lib().oracle_sobol_directions(_p(V))
    return V


def sobol_points(V, count: int) -> np.ndarray:
    """Points 0..count-1 of every dimension of the direction-number array V: [count, dims] uint32."""
    V = np.ascontiguousarray(V, dtype=np.uint32)
    out = np.zeros((count, V.shape[0]), np.uint32)
    L = lib()
    for d in range(V.shape[0]):
        row = np.ascontiguousarray(V[d])
        for q in range(count):
            out[q, d] = L.oracle_sobol_point(_p(row), q)
    return out


def qmc_scrambled(seed: int, replicate: int) -> np.ndarray:
    """Direction numbers of one replicate after the random linear scramble: [dims, 32]."""
    V = np.zeros((qmc_dims(), 32), np.uint32)
    lib().oracle_qmc_scrambled(int(seed), int(replicate), _p(V))
    return V


def qmc_shift(seed: int, entry: int, replicate: int, dim: int) -> int:
    return int(lib().oracle_qmc_shift(int(seed), int(entry), int(replicate), int(dim)))


def num_threads() -> int:
    return int(lib().oracle_num_threads())
