"""Sharding of the path sample over ranks (one process per GPU).

Paths are independent (Sec. 1; Sec. 7), so M paths per entry split into
disjoint index ranges, one per rank, with no data-path collective: rank r runs
paths [offset_r, offset_r + M_r) of every entry (the C-ABI's path_offset), and
the union over ranks is exactly the single-process sample of sum(M_r) paths.
The only exchange a merged estimate needs is per entry (M_r, mean_r, SE_r);
`merge` recombines them into the mean and standard error of the union
(sample mean and variance of Sec. 5, regrouped), in FP64 on the host.
"""
from __future__ import annotations

import numpy as np


def path_range(rank: int, world: int, paths: int) -> tuple[int, int]:
    """(path_offset, count) of rank `rank` when `paths` paths per entry are split
    over `world` ranks: contiguous blocks, the first `paths % world` ranks one longer."""
    if world < 1 or not 0 <= rank < world or paths < 0:
        raise ValueError("need 0 <= rank < world and paths >= 0")
    q, r = divmod(paths, world)
    count = q + (1 if rank < r else 0)
    offset = rank * q + min(rank, r)
    return offset, count


def merge(means, sems, counts):
    """Mean and standard error over the union of per-rank samples.

    means, sems: [ranks, entries]; counts: [ranks] paths per entry of each rank.
    With S1_r = M_r mean_r and S2_r = (M_r - 1) M_r SE_r^2 + M_r mean_r^2 (the
    per-rank sums of w and w^2), the union has mean S1/M and variance
    (S2 - M mean^2)/(M - 1), M = sum M_r; SE = sqrt(variance / M).
    """
    means = np.asarray(means, dtype=np.float64)
    sems = np.asarray(sems, dtype=np.float64)
    Mr = np.asarray(counts, dtype=np.float64).reshape(-1, 1)
    if means.shape != sems.shape or means.shape[0] != Mr.shape[0]:
        raise ValueError("means, sems and counts disagree in shape")
    M = float(Mr.sum())
    if M <= 0:
        raise ValueError("no paths")
    keep = Mr > 0
    s1 = np.where(keep, Mr * means, 0.0).sum(axis=0)
    s2 = np.where(keep, (Mr - 1.0) * Mr * sems * sems + Mr * means * means, 0.0).sum(axis=0)
    mean = s1 / M
    var = np.maximum((s2 - M * mean * mean) / (M - 1.0), 0.0) if M > 1 else np.zeros_like(mean)
    return mean, np.sqrt(var / M)
