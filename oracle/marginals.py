"""Log-domain application of the Gibbs kernel and the marginals of a returned
iterate, vectorised so that full-size workloads (2^23 points, 512 x 512 and
64^3 grids) can be checked entry by entry.

Test infrastructure only (see ``oracle/__init__.py``).

For potentials f = log u and g = log v (any magnitude, -inf allowed) the plan
of Algorithm 1 is P_ij = e^{f_i} K_ij e^{g_j} with K_ij = e^{-|i-j| h / eps}
(Section 2; Section 4 for the separable 2D kernel, and its closing remark for
a third axis).  Its marginals are
    P 1   = e^{f} * (K e^{g})        (the row marginal, = a after the u-update)
    P^T 1 = e^{g} * (K e^{f})        (the column marginal; K is symmetric)
and the stopping test of Algorithm 1 is || P^T 1 - b ||_1.

log(K e^f)_k = log sum_j e^{f_j - |k - j| c} (c = h / eps) is evaluated from
the definition, split by the sign of k - j so that each part is a running
log-sum-exp over j:
    sum_{j <= k} e^{f_j - (k - j) c} = e^{-k c} sum_{j <= k} e^{f_j + j c}
    sum_{j >  k} e^{f_j - (j - k) c} = e^{+k c} sum_{j >  k} e^{f_j - j c}
(an exact rearrangement of the same terms; numpy's logaddexp.accumulate forms
the running sums in FP64).  On a grid the kernel is the product of the axis
kernels, so the nD application is the 1D one along each axis in turn.
"""
from __future__ import annotations

from typing import Sequence

import numpy as np


def log_apply_1d(f, c: float, axis: int = -1) -> np.ndarray:
    """log(K e^f) along `axis` of f, K_kj = e^{-|k-j| c}.  -inf where the sum
    is zero."""
    f = np.moveaxis(np.asarray(f, dtype=np.float64), axis, -1)
    n = f.shape[-1]
    j = np.arange(n, dtype=np.float64) * c
    with np.errstate(invalid="ignore"):
        lower = np.logaddexp.accumulate(f + j, axis=-1) - j            # j <= k
        upper_incl = np.flip(np.logaddexp.accumulate(np.flip(f - j, -1), axis=-1), -1)
    upper = np.full_like(f, -np.inf)                                   # j > k
    upper[..., :-1] = upper_incl[..., 1:] + j[:-1]
    out = np.logaddexp(lower, upper)
    return np.moveaxis(out, -1, axis)


def log_apply(F, cs: Sequence[float]) -> np.ndarray:
    """log(K e^F) for the separable grid kernel.  F has shape (n,), (n_slow,
    n_fast) or (n_slow, n_mid, n_fast) (the fast axis contiguous, Section 4's
    first index); cs = (c_fast[, c_mid], c_slow) with c = h_axis / eps."""
    F = np.asarray(F, dtype=np.float64)
    assert len(cs) == F.ndim
    out = F
    for k, c in enumerate(cs):          # k = 0 is the fast (last) axis
        out = log_apply_1d(out, float(c), axis=F.ndim - 1 - k)
    return out


def row_marginal(f, g, cs) -> np.ndarray:
    """P 1 = e^f * (K e^g)."""
    return np.exp(np.asarray(f, dtype=np.float64) + log_apply(g, cs))


def col_marginal(f, g, cs) -> np.ndarray:
    """P^T 1 = e^g * (K e^f)."""
    return np.exp(np.asarray(g, dtype=np.float64) + log_apply(f, cs))


def marginal_error(f, g, b, cs) -> float:
    """|| P^T 1 - b ||_1, the quantity of Algorithm 1's while condition."""
    return float(np.abs(col_marginal(f, g, cs) - np.asarray(b, dtype=np.float64)).sum())
