"""Closed forms and brute force that pin the oracle from outside itself.

Test infrastructure only (see ``oracle/__init__.py``).
"""
from __future__ import annotations

import numpy as np


def w1_exact_1d(a, b, h: float) -> float:
    """Exact Wasserstein-1 between two histograms on a uniform 1D grid with
    spacing h: W1 = h * sum_k |A_k - B_k|, A, B the cumulative sums (the
    north-west-corner coupling is optimal for a convex cost on the line).
    This is the eps -> 0 limit of the value of eq. "kantorovich" that
    Algorithm 1 approximates."""
    A = np.cumsum(np.asarray(a, dtype=np.float64))
    B = np.cumsum(np.asarray(b, dtype=np.float64))
    return float(h * np.abs(A[:-1] - B[:-1]).sum())


def w1_lp(a, b, C) -> float:
    """Brute-force linear program of eq. "kantorovich" on the N x N coupling
    (scipy HiGHS): min <gamma, C> s.t. gamma 1 = a, gamma^T 1 = b, gamma >= 0."""
    from scipy.optimize import linprog
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    n, m = a.size, b.size
    A_eq = np.zeros((n + m, n * m))
    for i in range(n):
        A_eq[i, i * m:(i + 1) * m] = 1.0
    for j in range(m):
        A_eq[n + j, j::m] = 1.0
    res = linprog(np.asarray(C, dtype=np.float64).reshape(-1), A_eq=A_eq,
                  b_eq=np.concatenate([a, b]), bounds=(0, None), method="highs")
    assert res.status == 0, res.message
    return float(res.fun)


def entropy(p) -> float:
    """Shannon entropy -sum p log p (0 log 0 = 0)."""
    p = np.asarray(p, dtype=np.float64).reshape(-1)
    p = p[p > 0]
    return float(-(p * np.log(p)).sum())
