"""Multilevel Monte Carlo over the time step of the STRANG and LIE functionals
(Giles, Oper. Res. 56, 2008), on top of the level-difference estimator of the
C-ABI (mcx_estimate_level_difference).

The target is the split estimate with the finest step count N_L = n0 2^L:

    E[P_L] = E[P_0] + sum_{l=1..L} E[P_l - P_{l-1}],

level 0 the plain estimate with n0 steps, level l the coupled difference of the
functionals with N_l and N_l / 2 steps on the same paths.  The levels draw from
disjoint path ranges (path_offset = l 2^40), so they are independent and the
standard errors add in quadrature.  Sampling and the combination run in the
library's kernels (mcx_combine_levels adds the levels on the device); this
module only chooses sample sizes and path ranges.
"""
from __future__ import annotations

import math

LEVEL_STRIDE = 1 << 40  # path-index stride between levels


def allocation(variances, costs, eps: float) -> list[int]:
    """Samples per level minimising the cost for a sampling variance eps^2:
    M_l = ceil(eps^-2 sqrt(V_l / C_l) sum_k sqrt(V_k C_k)) (Giles 2008, Eq. (6)),
    V_l the per-sample variance and C_l the per-sample cost of level l."""
    if eps <= 0:
        raise ValueError("eps must be positive")
    if len(variances) != len(costs) or not variances:
        raise ValueError("one variance and one cost per level")
    total = sum(math.sqrt(max(v, 0.0) * c) for v, c in zip(variances, costs))
    return [max(1, math.ceil(math.sqrt(max(v, 0.0) / c) * total / eps ** 2)) for v, c in zip(variances, costs)]


def estimate(plan, v, t: float, n0: int, levels: int, paths, entries=None, seed: int = 0, mode: str = "strang",
             prec: str = "fp32"):
    """Multilevel estimate of the STRANG/LIE target with n0 * 2^levels steps.

    `paths` gives the samples per level (levels + 1 numbers).  Returns
    (mean, sem, per_level) with per_level a list of (mean, sem) tensors."""
    if mode not in ("strang", "lie"):
        raise ValueError("multilevel estimates need the STRANG or LIE functional")
    if n0 < 1 or levels < 0 or len(paths) != levels + 1:
        raise ValueError("need n0 >= 1 and one sample size per level")
    per_level = [plan.estimate(v, t, int(paths[0]), entries=entries, seed=seed, path_offset=0, mode=mode,
                               nsteps=n0, prec=prec)]
    for lvl in range(1, levels + 1):
        per_level.append(plan.estimate_level_difference(v, t, n0 << lvl, int(paths[lvl]), entries=entries,
                                                        seed=seed, path_offset=lvl * LEVEL_STRIDE, mode=mode,
                                                        prec=prec))
    mean, sem = plan.combine_levels([m for m, _ in per_level], [s for _, s in per_level])
    return mean, sem, per_level


PILOT_OFFSET = 1 << 39  # pilot samples of level l use paths l 2^40 + 2^39 + p (disjoint from the run's)


def adaptive(plan, v, t: float, n0: int, levels: int, eps: float, pilot_paths: int = 10000, costs=None,
             entries=None, seed: int = 0, mode: str = "strang", prec: str = "fp32"):
    """Giles' multilevel method with a pilot: per level, `pilot_paths` samples give the
    per-sample variance V_l (mean over the entries of M SE^2); the allocation for a
    sampling error eps (per entry, root mean square over entries) uses the costs
    C_l (default: equal, since a walker's cost does not depend on the step count);
    then the multilevel estimate with those sample sizes on fresh paths.
    Returns (mean, sem, per_level, sizes)."""
    if mode not in ("strang", "lie"):
        raise ValueError("multilevel estimates need the STRANG or LIE functional")
    if pilot_paths < 2:
        raise ValueError("the pilot needs at least two samples per level")
    V = []
    for lvl in range(levels + 1):
        off = lvl * LEVEL_STRIDE + PILOT_OFFSET
        if lvl == 0:
            _, s = plan.estimate(v, t, int(pilot_paths), entries=entries, seed=seed, path_offset=off, mode=mode,
                                 nsteps=n0, prec=prec)
        else:
            _, s = plan.estimate_level_difference(v, t, n0 << lvl, int(pilot_paths), entries=entries, seed=seed,
                                                  path_offset=off, mode=mode, prec=prec)
        V.append(float((s * s).mean()) * pilot_paths)
    C = list(costs) if costs is not None else [1.0] * (levels + 1)
    sizes = allocation(V, C, eps)
    if max(sizes) > PILOT_OFFSET:
        raise ValueError("the allocation exceeds 2^39 samples on a level")
    mean, sem, per_level = estimate(plan, v, t, n0, levels, sizes, entries=entries, seed=seed, mode=mode, prec=prec)
    return mean, sem, per_level, sizes
