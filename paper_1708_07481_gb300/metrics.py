"""Partition quality reported beside the timings: PM, PR, PP (Sec. IV reports them for every
run; the paper defines them by reference to the Graph Challenge).

- PM: the best one-to-one matching of true and found blocks (Hungarian assignment on the
  contingency table), matched vertices / n.
- PR: pairwise recall, pairs placed together in both / pairs together in the truth.
- PP: pairwise precision, pairs placed together in both / pairs together in the answer.

Host-side reporting only: nothing here feeds the partition itself.
"""
from __future__ import annotations

import numpy as np
from scipy.optimize import linear_sum_assignment


def contingency(truth: np.ndarray, found: np.ndarray) -> np.ndarray:
    truth = np.asarray(truth, dtype=np.int64)
    found = np.asarray(found, dtype=np.int64)
    t = truth.max() + 1 if truth.size else 0
    f = found.max() + 1 if found.size else 0
    c = np.zeros((t, f), dtype=np.int64)
    np.add.at(c, (truth, found), 1)
    return c


def pm_pr_pp(truth: np.ndarray, found: np.ndarray) -> tuple[float, float, float]:
    c = contingency(truth, found)
    n = int(c.sum())
    if n == 0:
        return 1.0, 1.0, 1.0
    rows, cols = linear_sum_assignment(-c)
    pm = float(c[rows, cols].sum()) / n

    def pairs(x):
        x = x.astype(np.float64)
        return float((x * (x - 1) / 2).sum())

    both = pairs(c)
    tt = pairs(c.sum(axis=1))
    ff = pairs(c.sum(axis=0))
    pr = both / tt if tt > 0 else 1.0
    pp = both / ff if ff > 0 else 1.0
    return pm, pr, pp
