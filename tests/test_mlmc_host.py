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


class _FakePlan:
    """Records the calls the driver makes and returns fixed per-level results."""

    def __init__(self):
        self.calls = []

    def estimate(self, v, t, paths, entries=None, seed=0, path_offset=0, mode="exact", nsteps=1, prec="fp32"):
        import torch

        self.calls.append(("plain", nsteps, paths, path_offset, mode, seed))
        return torch.tensor([10.0, 20.0]), torch.tensor([0.3, 0.4])

    def estimate_level_difference(self, v, t, nsteps, paths, entries=None, seed=0, path_offset=0, mode="strang",
                                  prec="fp32"):
        import torch

        self.calls.append(("diff", nsteps, paths, path_offset, mode, seed))
        return torch.tensor([0.1 * nsteps, -0.01 * nsteps]), torch.tensor([0.01, 0.02])

    def combine_levels(self, means, sems):
        """Stands in for the library's device combination (checked on the GPU)."""
        import torch

        self.calls.append(("combine", len(means)))
        return torch.stack(means).sum(dim=0), torch.stack([s * s for s in sems]).sum(dim=0).sqrt()


def test_driver_levels_offsets_and_combination():
    torch = pytest.importorskip("torch")
    plan = _FakePlan()
    mean, sem, levels = mlmc.estimate(plan, None, 0.5, 4, 3, [1000, 500, 250, 125], seed=7, mode="lie")
    assert plan.calls == [("plain", 4, 1000, 0, "lie", 7), ("diff", 8, 500, mlmc.LEVEL_STRIDE, "lie", 7),
                          ("diff", 16, 250, 2 * mlmc.LEVEL_STRIDE, "lie", 7),
                          ("diff", 32, 125, 3 * mlmc.LEVEL_STRIDE, "lie", 7), ("combine", 4)]
    assert torch.allclose(mean, torch.tensor([10.0 + 0.1 * (8 + 16 + 32), 20.0 - 0.01 * (8 + 16 + 32)]))
    assert torch.allclose(sem, torch.tensor([math.sqrt(0.09 + 3e-4), math.sqrt(0.16 + 3 * 4e-4)]))
    assert len(levels) == 4


def test_driver_rejects_exact_and_bad_sizes():
    pytest.importorskip("torch")
    with pytest.raises(ValueError):
        mlmc.estimate(_FakePlan(), None, 0.5, 4, 1, [10, 10], mode="exact")
    with pytest.raises(ValueError):
        mlmc.estimate(_FakePlan(), None, 0.5, 4, 2, [10, 10])


def test_adaptive_pilot_then_allocation():
    torch = pytest.importorskip("torch")
    plan = _FakePlan()
    mean, sem, levels, sizes = mlmc.adaptive(plan, None, 0.5, 2, 2, eps=0.01, pilot_paths=100, seed=3)
    pilot, run = plan.calls[:3], plan.calls[3:]
    assert [c[0] for c in pilot] == ["plain", "diff", "diff"] and [c[1] for c in pilot] == [2, 4, 8]
    assert all(c[2] == 100 for c in pilot)
    assert [c[3] for c in pilot] == [mlmc.PILOT_OFFSET, mlmc.LEVEL_STRIDE + mlmc.PILOT_OFFSET,
                                     2 * mlmc.LEVEL_STRIDE + mlmc.PILOT_OFFSET]
    # pilot variances: mean SE^2 x 100 -> level 0: (0.09 + 0.16)/2 x 100, levels 1, 2: (1e-4 + 4e-4)/2 x 100
    V = [12.5, 0.025, 0.025]
    assert sizes == mlmc.allocation(V, [1.0, 1.0, 1.0], 0.01)
    assert run[-1] == ("combine", 3)
    run = run[:-1]
    assert [c[2] for c in run] == sizes and [c[3] for c in run] == [0, mlmc.LEVEL_STRIDE, 2 * mlmc.LEVEL_STRIDE]
    with pytest.raises(ValueError):
        mlmc.adaptive(plan, None, 0.5, 2, 2, eps=0.01, pilot_paths=1)
