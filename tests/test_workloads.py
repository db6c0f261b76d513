"""Input generators: structure of the seeded synthetic matrices (they hold none of
the method's arithmetic; both the oracle and the GPU path read them as data)."""
import numpy as np

import workloads as W


def _check_csr(c, symmetric=True):
    assert c.row_ptr[0] == 0 and c.row_ptr[-1] == c.nnz and np.all(np.diff(c.row_ptr) >= 0)
    for i in range(0, c.n, max(1, c.n // 50)):
        cols = c.col[c.row_ptr[i]:c.row_ptr[i + 1]]
        assert np.all(np.diff(cols) > 0) and not np.any(cols == i)
    if symmetric:
        a = c.to_scipy()
        assert (a != a.T).nnz == 0


def test_small_world_structure():
    c = W.small_world(20000, 1, 0.2, 3)
    _check_csr(c)
    deg = np.diff(c.row_ptr)
    assert deg.min() >= 2 and abs(deg.mean() - 2.4) < 0.02
    a = c.to_scipy().tolil()
    assert all(a[i, (i + 1) % 20000] == 1 for i in range(0, 20000, 997))  # the ring is present
    c2 = W.small_world(20000, 2, 0.0, 3)  # no shortcuts: the 2-nearest-neighbour ring
    assert np.all(np.diff(c2.row_ptr) == 4)
    assert np.array_equal(W.small_world(5000, 1, 0.2, 9).col, W.small_world(5000, 1, 0.2, 9).col)


def test_erdos_renyi_and_barabasi_albert_structure():
    e = W.erdos_renyi(20000, 10, 1)
    _check_csr(e)
    assert abs(e.nnz / e.n - 10) < 0.3
    b = W.barabasi_albert(20000, 5, 1)
    _check_csr(b)
    deg = np.diff(b.row_ptr)
    assert deg.min() >= 5 and deg.max() > 100  # preferential attachment grows hubs
