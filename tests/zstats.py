"""Statistical agreement of Monte Carlo estimates with their exact targets.

The estimates are random, so correctness is decided on per-entry z-scores
z_i = (xhat_i - x_i) / SE_i over k entries, by three bounds:
  (i)   the fraction with |z| > 3 is at most p + 5 sqrt(p / k), p the two-sided
        tail probability of |z| > 3 (0.0027 for a normal z);
  (ii)  |mean z| <= 5 sqrt(s2 / k), s2 the variance of z (1 for a normal z);
  (iii) var z within [0.8, 1.25] s2, checked when every entry has at least 1000
        paths (or replicates) and k >= 100, so that the spread is well estimated.
When the standard error comes from only R replicate means (randomised QMC), z
follows Student's t with R - 1 degrees of freedom: p and s2 are taken from it.
"""
import math

import numpy as np


def _t_tail3(dof):
    """P(|T| > 3) for Student's t with `dof` degrees of freedom (regularised incomplete beta)."""
    from scipy import stats

    return float(2 * stats.t.sf(3.0, dof))


def check(z, samples=None, dof=None):
    """Assert the three bounds on z (array of z-scores); `samples` the paths (or
    replicates) per entry, `dof` the degrees of freedom of a replicate SE.
    Returns z."""
    z = np.asarray(z, dtype=np.float64)
    k = z.size
    if dof is None:
        p, s2 = 0.0027, 1.0
    else:
        p, s2 = _t_tail3(dof), dof / (dof - 2.0)
    frac = float((np.abs(z) > 3).mean())
    assert frac <= p + 5 * math.sqrt(p / k), ("tail", frac, p, k)
    assert abs(float(z.mean())) <= 5 * math.sqrt(s2 / k), ("mean", float(z.mean()), k)
    if samples is not None and samples >= 1000 and k >= 100:
        assert 0.8 * s2 <= float(z.var()) <= 1.25 * s2, ("var", float(z.var()), s2)
    return z
