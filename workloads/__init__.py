"""Seeded synthetic inputs for the Monte Carlo exp(tA)v estimator.

This module only builds inputs: sparse matrices in CSR form (int64 row
pointers, int32 sorted column indices, float64 values), starting vectors and
entry sets.  It holds none of the estimator's arithmetic, so both the CUDA
library and the CPU oracle may consume what it returns.

Every generator takes an explicit seed and uses numpy's PCG64 stream, so the
same call gives the same arrays on any machine.

Workload shapes follow the problem classes the paper studies (Sec. 2: A
symmetric with a Laplacian part; Sec. 6: small-world / scale-free networks)
plus PDE and CTMC generators:

* ``grid_laplacian_2d`` / ``grid_laplacian_3d``: Dirichlet finite-difference
  Laplacians (5- and 7-point), the method-of-lines case of Sec. 1.
* ``erdos_renyi``: symmetric 0/1 adjacency of G(n, p).
* ``barabasi_albert``: symmetric 0/1 adjacency of a preferential-attachment
  graph (the scale-free networks of Sec. 6).
* ``random_generator``: CTMC generators Q (rows sum to zero, lognormal rates),
  the transient-analysis case of Sec. 1.
"""
from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass
class CSR:
    """A square sparse matrix in CSR form with sorted, unique columns per row."""

    n: int
    row_ptr: np.ndarray  # int64 [n+1]
    col: np.ndarray  # int32 [nnz]
    val: np.ndarray  # float64 [nnz]

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def to_dense(self) -> np.ndarray:
        d = np.zeros((self.n, self.n), dtype=np.float64)
        rows = np.repeat(np.arange(self.n), np.diff(self.row_ptr))
        d[rows, self.col] = self.val
        return d

    def to_scipy(self):
        import scipy.sparse as sp

        return sp.csr_matrix((self.val, self.col, self.row_ptr), shape=(self.n, self.n))


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def from_coo(n: int, rows: np.ndarray, cols: np.ndarray, vals: np.ndarray) -> CSR:
    """Assemble CSR from COO triplets (duplicates are summed, columns sorted)."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    vals = np.asarray(vals, dtype=np.float64)
    key = rows * n + cols
    order = np.argsort(key, kind="stable")
    key = key[order]
    vals = vals[order]
    uniq, start = np.unique(key, return_index=True)
    summed = np.add.reduceat(vals, start) if len(vals) else vals
    r = uniq // n
    c = uniq % n
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(row_ptr, r + 1, 1)
    row_ptr = np.cumsum(row_ptr)
    return CSR(n, row_ptr, c.astype(np.int32), summed.astype(np.float64))


def dense_to_csr(a: np.ndarray) -> CSR:
    a = np.asarray(a, dtype=np.float64)
    r, c = np.nonzero(a)
    return from_coo(a.shape[0], r, c, a[r, c])


# ---------------------------------------------------------------------------
# PDE operators
# ---------------------------------------------------------------------------

def grid_laplacian_2d(m: int) -> CSR:
    """5-point Dirichlet Laplacian on an m x m interior grid, h = 1/(m+1).

    Unknown (ix, iy) has row index iy*m + ix.  Off-diagonals are 1/h^2, the
    diagonal is -4/h^2.
    """
    h2inv = float((m + 1) ** 2)
    n = m * m
    idx = np.arange(n, dtype=np.int64).reshape(m, m)  # [iy, ix]
    rows, cols, vals = [idx.ravel()], [idx.ravel()], [np.full(n, -4.0 * h2inv)]
    for d in ((0, 1), (0, -1), (1, 0), (-1, 0)):
        sl_src = tuple(slice(max(0, -k), m - max(0, k)) for k in d)
        sl_dst = tuple(slice(max(0, k), m + min(0, k)) for k in d)
        rows.append(idx[sl_src].ravel())
        cols.append(idx[sl_dst].ravel())
        vals.append(np.full(idx[sl_src].size, h2inv))
    return _csr_from_sorted_rows(n, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))


def grid_laplacian_3d(m: int) -> CSR:
    """7-point Dirichlet Laplacian on an m^3 interior grid, h = 1/(m+1).

    Unknown (ix, iy, iz) has row index (iz*m + iy)*m + ix.
    """
    h2inv = float((m + 1) ** 2)
    n = m ** 3
    idx = np.arange(n, dtype=np.int64).reshape(m, m, m)  # [iz, iy, ix]
    rows, cols, vals = [idx.ravel()], [idx.ravel()], [np.full(n, -6.0 * h2inv)]
    for d in ((0, 0, 1), (0, 0, -1), (0, 1, 0), (0, -1, 0), (1, 0, 0), (-1, 0, 0)):
        sl_src = tuple(slice(max(0, -k), m - max(0, k)) for k in d)
        sl_dst = tuple(slice(max(0, k), m + min(0, k)) for k in d)
        rows.append(idx[sl_src].ravel())
        cols.append(idx[sl_dst].ravel())
        vals.append(np.full(idx[sl_src].size, h2inv))
    return _csr_from_sorted_rows(n, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))


def _csr_from_sorted_rows(n, rows, cols, vals) -> CSR:
    """COO -> CSR for triplets with no duplicates (faster than from_coo)."""
    order = np.lexsort((cols, rows))
    rows = rows[order]
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=n), out=row_ptr[1:])
    return CSR(n, row_ptr, cols[order].astype(np.int32), vals[order].astype(np.float64))


# ---------------------------------------------------------------------------
# Networks
# ---------------------------------------------------------------------------

def _symmetric_adjacency(n: int, a: np.ndarray, b: np.ndarray) -> CSR:
    """0/1 symmetric adjacency from an undirected edge list (a != b, unique)."""
    rows = np.concatenate([a, b]).astype(np.int64)
    cols = np.concatenate([b, a]).astype(np.int64)
    return _csr_from_sorted_rows(n, rows, cols, np.ones(rows.size))


def erdos_renyi(n: int, mean_degree: float, seed: int) -> CSR:
    """Symmetric 0/1 adjacency of G(n, p), p = mean_degree/(n-1), no self-loops.

    The edge count is drawn Binomial(n(n-1)/2, p); that many distinct
    unordered pairs are then drawn uniformly.
    """
    rng = _rng(seed)
    pairs = n * (n - 1) // 2
    p = mean_degree / (n - 1)
    m = int(rng.binomial(pairs, p))
    keys = np.empty(0, dtype=np.int64)
    while keys.size < m:
        need = int((m - keys.size) * 1.05) + 16
        i = rng.integers(0, n, size=need, dtype=np.int64)
        j = rng.integers(0, n, size=need, dtype=np.int64)
        keep = i != j
        lo = np.minimum(i, j)[keep]
        hi = np.maximum(i, j)[keep]
        keys = np.unique(np.concatenate([keys, lo * n + hi]))
    if keys.size > m:
        keys = rng.choice(keys, size=m, replace=False)
    return _symmetric_adjacency(n, keys // n, keys % n)


def small_world(n: int, k: int, p: float, seed: int) -> CSR:
    """Symmetric 0/1 adjacency of a small-world graph in the style of the
    Watts-Strogatz model without rewiring: the ring lattice joining each node to
    its k nearest neighbours on each side, plus, for each node with
    probability p, one shortcut to a node drawn uniformly among the others
    (duplicates of existing edges are dropped).  Mean degree about 2k + 2p.
    """
    rng = _rng(seed)
    i = np.arange(n, dtype=np.int64)
    lo_l, hi_l = [], []
    for j in range(1, k + 1):
        u, v = i, (i + j) % n
        lo_l.append(np.minimum(u, v))
        hi_l.append(np.maximum(u, v))
    has = rng.random(n) < p
    src = i[has]
    dst = rng.integers(0, n - 1, size=src.size, dtype=np.int64)
    dst = dst + (dst >= src)  # uniform over the other nodes
    lo_l.append(np.minimum(src, dst))
    hi_l.append(np.maximum(src, dst))
    keys = np.unique(np.concatenate(lo_l) * n + np.concatenate(hi_l))
    return _symmetric_adjacency(n, keys // n, keys % n)


def barabasi_albert(n: int, m: int, seed: int) -> CSR:
    """Symmetric 0/1 adjacency of a Barabasi-Albert graph.

    Seed graph: the clique on nodes 0..m.  Each later node t attaches m edges
    to distinct earlier nodes, each chosen with probability proportional to
    degree: a uniform position in the list of edge endpoints present when t
    arrives (each edge contributes both endpoints).  Draws that repeat a
    target of the same node are redrawn.
    """
    rng = _rng(seed)
    m0 = m + 1
    seed_a, seed_b = np.triu_indices(m0, k=1)
    e_seed = seed_a.size
    n_new = n - m0
    if n_new <= 0:
        return _symmetric_adjacency(n, seed_a, seed_b)
    # Edge e (0-based over all edges) has endpoint list positions 2e (first) and 2e+1 (second).
    # Seed edges: first = seed_a, second = seed_b.  New edges of node t: first = t, second = target.
    t_of = np.repeat(np.arange(m0, n, dtype=np.int64), m)  # node adding each new edge
    ne = t_of.size
    # endpoint-list length seen by node t: 2 * (edges present before t)
    len_t = 2 * (e_seed + (t_of - m0) * m)
    pos = (rng.random(ne) * len_t).astype(np.int64)
    pos = np.minimum(pos, len_t - 1)

    def resolve(pos):
        """Map endpoint-list positions to node ids (pointer jumping to earlier edges)."""
        node = np.full(ne, -1, dtype=np.int64)
        cur = pos.copy()
        todo = np.arange(ne)
        while todo.size:
            p = cur[todo]
            e = p // 2
            first = (p % 2) == 0
            is_seed = e < e_seed
            # seed edges: known endpoints
            s = is_seed
            node[todo[s]] = np.where(first[s], seed_a[e[s] % max(e_seed, 1)], seed_b[e[s] % max(e_seed, 1)])
            # new edges, first endpoint: the node that added it
            f = (~is_seed) & first
            node[todo[f]] = t_of[e[f] - e_seed]
            # new edges, second endpoint: follow that edge's own position
            g = (~is_seed) & (~first)
            cur[todo[g]] = pos[e[g] - e_seed]
            todo = todo[g]
        return node

    for _ in range(1000):
        tgt = resolve(pos)
        blk = tgt.reshape(-1, m)
        srt = np.sort(blk, axis=1)
        dup_rows = np.nonzero((srt[:, 1:] == srt[:, :-1]).any(axis=1))[0]
        if dup_rows.size == 0:
            break
        # redraw every edge after the first occurrence of a repeated target
        for r in dup_rows:
            seen = set()
            for k in range(m):
                e = r * m + k
                if int(blk[r, k]) in seen:
                    pos[e] = min(int(rng.random() * len_t[e]), int(len_t[e]) - 1)
                seen.add(int(blk[r, k]))
    else:  # pragma: no cover
        raise RuntimeError("barabasi_albert: could not draw distinct targets")
    a = np.concatenate([seed_a, t_of])
    b = np.concatenate([seed_b, tgt])
    return _symmetric_adjacency(n, a, b)


# ---------------------------------------------------------------------------
# CTMC generators
# ---------------------------------------------------------------------------

def random_generator(n: int, seed: int, kmin: int = 8, kmax: int = 32) -> CSR:
    """Random CTMC generator Q: per row k ~ U{kmin..kmax} distinct off-diagonal
    columns, rates exp(N(0,1)), diagonal = -(row sum of off-diagonals)."""
    rng = _rng(seed)
    k = rng.integers(kmin, kmax + 1, size=n)
    kcap = min(kmax, n - 1)
    k = np.minimum(k, kcap)
    ncand = min(n - 1, kmax + 24)
    rows_l, cols_l = [], []
    todo = np.arange(n)
    while todo.size:
        cand = rng.integers(0, n - 1, size=(todo.size, ncand), dtype=np.int64)
        cand = cand + (cand >= todo[:, None])  # skip the diagonal
        srt = np.sort(cand, axis=1)
        uniq = np.ones_like(srt, dtype=bool)
        uniq[:, 1:] = srt[:, 1:] != srt[:, :-1]
        cnt = uniq.sum(axis=1)
        ok = cnt >= k[todo]
        for_rows = todo[ok]
        s_ok = srt[ok]
        u_ok = uniq[ok]
        # choose k of the distinct values uniformly: random keys, keep the k smallest
        keys = rng.random(s_ok.shape)
        keys[~u_ok] = 2.0
        sel = np.argsort(keys, axis=1)
        kk = k[for_rows]
        take = np.arange(s_ok.shape[1])[None, :] < kk[:, None]
        chosen = np.take_along_axis(s_ok, sel, axis=1)
        rows_l.append(np.repeat(for_rows, kk))
        cols_l.append(chosen[take])
        todo = todo[~ok]
    rows = np.concatenate(rows_l)
    cols = np.concatenate(cols_l)
    rates = np.exp(rng.standard_normal(rows.size))
    off = _csr_from_sorted_rows(n, rows, cols, rates)
    # diagonal = -(row sum of the off-diagonal rates, summed left to right in column
    # order), so that every row of Q sums to exactly 0 in floating point too
    deg = np.diff(off.row_ptr)
    acc = np.zeros(n)
    for k in range(int(deg.max()) if n else 0):
        has = deg > k
        acc[has] += off.val[off.row_ptr[:-1][has] + k]
    rows = np.concatenate([np.repeat(np.arange(n), deg), np.arange(n)])
    cols = np.concatenate([off.col.astype(np.int64), np.arange(n)])
    vals = np.concatenate([off.val, -acc])
    return _csr_from_sorted_rows(n, rows, cols, vals)


def transpose(a: CSR) -> CSR:
    rows = np.repeat(np.arange(a.n, dtype=np.int64), np.diff(a.row_ptr))
    return _csr_from_sorted_rows(a.n, a.col.astype(np.int64), rows, a.val.copy())


# ---------------------------------------------------------------------------
# Vectors and entry sets
# ---------------------------------------------------------------------------

def uniform_vector(n: int, seed: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    return _rng(seed).uniform(lo, hi, size=n)


def gaussian_bump_3d(m: int, seed: int, width: float = 0.1, noise: float = 1e-3) -> np.ndarray:
    """exp(-|x-c|^2/(2 width^2)) + noise*U[0,1) on the interior grid x = (i+1)h."""
    h = 1.0 / (m + 1)
    g = (np.arange(m) + 1) * h - 0.5
    z, y, x = np.meshgrid(g, g, g, indexing="ij")
    bump = np.exp(-(x * x + y * y + z * z) / (2.0 * width * width)).ravel()
    return bump + noise * _rng(seed).random(m ** 3)


def dirichlet_probability(n: int, seed: int) -> np.ndarray:
    """Flat-Dirichlet probability vector (normalised Exp(1) draws)."""
    e = _rng(seed).exponential(1.0, size=n)
    return e / e.sum()


def random_entries(n: int, k: int, seed: int) -> np.ndarray:
    """k distinct entry indices drawn uniformly from 0..n-1 (int32, sorted)."""
    return np.sort(_rng(seed).choice(n, size=k, replace=False)).astype(np.int32)


def ctmc_batch(count: int, seed: int, n_min: int = 1000, n_max: int = 100000, times=(0.1, 1.0, 10.0),
               paths_per_state: int = 64):
    """Batched CTMC transients: `count` random generators with sizes drawn
    log-uniformly in [n_min, n_max], each with a flat-Dirichlet start vector,
    the given horizons and paths_per_state * n forward paths per horizon.

    Returns a list of dicts (row_ptr, col, val, v, times, paths, csr)."""
    rng = _rng(seed)
    sizes = np.rint(10.0 ** rng.uniform(np.log10(n_min), np.log10(n_max), size=count)).astype(np.int64)
    out = []
    for b, n in enumerate(sizes):
        q = random_generator(int(n), seed * 100003 + 2 * b)
        p0 = dirichlet_probability(int(n), seed * 100003 + 2 * b + 1)
        out.append({"row_ptr": q.row_ptr, "col": q.col, "val": q.val, "v": p0,
                    "times": np.asarray(times, dtype=np.float64), "paths": int(paths_per_state * n), "csr": q})
    return out
