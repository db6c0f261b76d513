"""Host logic of the multilevel driver: Giles' sample allocation."""
import math

import pytest

from paper_1904_12759_gb300 import mlmc


def test_allocation_proportional_to_sqrt_v_over_c_and_meets_the_variance():
    V = [1.0, 0.25, 0.0625, 0.015625]
    C = [1.0, 1.0, 2.0, 4.0]
    eps = 1e-2
    M = mlmc.allocation(V, C, eps)
    # M_l / M_0 = sqrt(V_l / C_l) / sqrt(V_0 / C_0) up to the ceiling
    for m, v, c in zip(M, V, C):
        assert abs(m / M[0] - math.sqrt(v / c)) <= 1.0 / M[0] + 1e-12
    assert sum(v / m for v, m in zip(V, M)) <= eps ** 2 * (1 + 1e-12)
    # minimality: the continuous optimum's cost, sum sqrt(V C) squared / eps^2
    opt = sum(math.sqrt(v * c) for v, c in zip(V, C)) ** 2 / eps ** 2
    assert sum(m * c for m, c in zip(M, C)) <= opt + sum(C)


def test_allocation_rejects_bad_input():
    with pytest.raises(ValueError):
        mlmc.allocation([1.0], [1.0], 0.0)
    with pytest.raises(ValueError):
        mlmc.allocation([1.0, 2.0], [1.0], 0.1)
