"""isim_K (Sec. 6, Tables 1 and 3) against its definition evaluated with explicit sets."""
import numpy as np
import pytest

from paper_1904_12759_gb300 import metrics


def _brute(x, y, K):
    rx, ry = metrics.ranking(x), metrics.ranking(y)
    return sum(len(set(rx[:i]) ^ set(ry[:i])) / (2 * i) for i in range(1, K + 1)) / K


def test_isim_matches_set_definition():
    rng = np.random.default_rng(0)
    for n in (1, 2, 7, 50):
        x = rng.normal(size=n)
        y = x + rng.normal(scale=0.3, size=n)
        for K in {1, max(1, n // 10), n}:
            assert abs(metrics.isim(x, y, K) - _brute(x, y, K)) < 1e-14


def test_isim_limits_and_ties():
    x = np.arange(10.0)
    assert metrics.isim(x, x) == 0.0
    assert metrics.isim(x, 2 * x + 1) == 0.0  # only the ranking matters
    # reversed: the top-i sets are disjoint for i <= n/2
    assert abs(metrics.isim(x, -x, 5) - 1.0) < 1e-15
    assert metrics.isim(x, -x) == pytest.approx(_brute(x, -x, 10))
    # ties are broken by index on both sides
    assert metrics.isim(np.ones(6), np.ones(6)) == 0.0
    with pytest.raises(ValueError):
        metrics.isim(x, x, 0)
