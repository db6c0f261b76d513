"""Ranking similarity of communicability vectors (Sec. 6, the intersection
similarity used to compare node rankings; Tables 1 and 3).

For two score vectors x, y over the same nodes, let X_i and Y_i be the sets of
the i highest-scored nodes of each (ties broken by node index).  Then
    isim_K(x, y) = (1/K) sum_{i=1..K} |X_i symmetric-difference Y_i| / (2 i),
0 for identical top-K rankings and 1 for disjoint ones.  Since
|X_i sym-diff Y_i| = 2 i - 2 |X_i intersect Y_i|, one pass that grows both sets
by one node per step and counts the intersection gives every term in O(1).
Host-side analysis of estimates the library computed (numpy only).
"""
from __future__ import annotations

import numpy as np


def ranking(x) -> np.ndarray:
    """Node indices by decreasing score, ties by increasing index."""
    x = np.asarray(x, dtype=np.float64)
    return np.lexsort((np.arange(x.size), -x))


def isim(x, y, K: int | None = None) -> float:
    """Intersection similarity of the top-K rankings of x and y (K defaults to all nodes)."""
    rx, ry = ranking(x), ranking(y)
    n = rx.size
    if ry.size != n:
        raise ValueError("x and y must have the same length")
    K = n if K is None else int(K)
    if not 1 <= K <= n:
        raise ValueError("need 1 <= K <= n")
    in_x = np.zeros(n, dtype=bool)
    in_y = np.zeros(n, dtype=bool)
    inter = 0
    total = 0.0
    for i in range(K):
        a, b = rx[i], ry[i]
        in_x[a] = True
        if in_y[a]:
            inter += 1
        in_y[b] = True
        if in_x[b]:
            inter += 1
        total += 1.0 - inter / (i + 1)
    return total / K
