"""Pins of oracle/marginals.py (no GPU): the vectorised log-domain kernel
application against the O(N^2) definition summed term by term in log space,
against the log-domain recurrences of Section 3, and the marginals of an
oracle run against Algorithm 1's own invariants (exact row marginal after the
u-update; the reported marginal error)."""
import numpy as np
import pytest
from scipy.special import logsumexp

from oracle import cref, dense, marginals, recurrence
from paper_2202_10042_gb300 import inputs


def _brute_log_apply(F, hs, eps):
    """log sum_j exp(F_j - C_kj / eps) from the dense cost matrix."""
    F = np.asarray(F, dtype=np.float64)
    if F.ndim == 1:
        C = dense.ground_cost_1d(F.size, hs[0])
    elif F.ndim == 2:
        C = dense.ground_cost_2d(F.shape[1], F.shape[0], hs[0], hs[1])
    else:
        C = dense.ground_cost_3d(F.shape[2], F.shape[1], F.shape[0], hs[0], hs[1], hs[2])
    x = F.reshape(-1)
    return logsumexp(x[None, :] - C / eps, axis=1).reshape(F.shape)


@pytest.mark.parametrize("n", [1, 2, 3, 17, 64])
@pytest.mark.parametrize("c", [1e-3, 0.37, 6.0])
def test_log_apply_1d_equals_definition(n, c):
    rng = np.random.default_rng(n * 7 + int(c * 100))
    f = rng.normal(0.0, 30.0, n)
    if n > 4:
        f[[1, n - 2]] = -np.inf
    got = marginals.log_apply(f, [c])
    ref = _brute_log_apply(f, [c], 1.0)
    fin = np.isfinite(ref)
    assert np.array_equal(fin, np.isfinite(got))
    assert np.max(np.abs(got[fin] - ref[fin])) < 1e-11 * max(1.0, np.max(np.abs(ref[fin])))


def test_log_apply_1d_equals_lse_recurrence():
    rng = np.random.default_rng(3)
    f = np.cumsum(rng.normal(0, 0.3, 500)) * 40.0
    c = 0.02
    R, S = recurrence.lse_matvec(f, c)
    ref = np.logaddexp(R, S)
    got = marginals.log_apply_1d(f, c)
    assert np.max(np.abs(got - ref)) < 1e-9 * np.max(np.abs(ref))


@pytest.mark.parametrize("shape,hs", [((6, 9), (0.1, 0.3)), ((1, 7), (0.2, 0.5)), ((5, 1), (0.2, 0.05))])
def test_log_apply_2d_equals_definition(shape, hs):
    rng = np.random.default_rng(sum(shape))
    F = rng.normal(0.0, 5.0, shape)
    eps = 0.07
    got = marginals.log_apply(F, [hs[0] / eps, hs[1] / eps])
    ref = _brute_log_apply(F, hs, eps)
    assert np.max(np.abs(got - ref)) < 1e-11 * np.max(np.abs(ref))


def test_log_apply_3d_equals_definition():
    rng = np.random.default_rng(11)
    F = rng.normal(0.0, 5.0, (3, 4, 5))
    hs, eps = (0.1, 0.2, 0.3), 0.09
    got = marginals.log_apply(F, [h / eps for h in hs])
    ref = _brute_log_apply(F, hs, eps)
    assert np.max(np.abs(got - ref)) < 1e-11 * np.max(np.abs(ref))


def test_log_apply_large_offsets():
    """Potentials of magnitude 1e4 over 2^16 points (the scale of eps = 1e-4)
    stay finite and agree with the recurrence form."""
    rng = np.random.default_rng(5)
    n = 1 << 16
    f = -1e4 * np.abs(np.sin(np.linspace(0, 7, n))) + rng.normal(0, 1, n)
    c = 0.015
    got = marginals.log_apply_1d(f, c)
    assert np.all(np.isfinite(got))
    R, S = recurrence.lse_matvec(f[:4000], c)
    # the first 4000 entries depend on later points only through terms
    # smaller than e^{-c * (n - 4000) + 1e4}; compare away from the cut
    part = marginals.log_apply_1d(f[:4000], c)
    assert np.max(np.abs(part - np.logaddexp(R, S))) < 1e-8 * np.max(np.abs(part))


def test_marginals_of_an_oracle_run():
    """After Algorithm 1's u-update the row marginal is a; the column
    marginal's L1 distance to b is the error the oracle reports."""
    p = inputs.workload2(2, n=3000, eps=3e-3, itr_max=60)
    r = cref.solve(p.a, p.b, p.h[0], p.eps, 0.0, p.itr_max, tau=1e10, potentials=True)
    c = p.h[0] / p.eps
    row = marginals.row_marginal(r.f, r.g, [c])
    assert np.max(np.abs(row - p.a) / p.a) < 1e-11
    err = marginals.marginal_error(r.f, r.g, p.b, [c])
    assert abs(err - r.err) <= 1e-9 * r.err + 1e-12   # FP64 rounding of a unit mass


def test_marginals_of_a_2d_oracle_run():
    p = inputs.workload4(3, side=40, itr_max=30)
    r = cref.solve(p.a, p.b, p.h, p.eps, 0.0, p.itr_max, tau=1e10, potentials=True)
    cs = [p.h[0] / p.eps, p.h[1] / p.eps]
    row = marginals.row_marginal(r.f, r.g, cs)
    assert np.max(np.abs(row - p.a) / p.a) < 1e-11
    err = marginals.marginal_error(r.f, r.g, p.b, cs)
    assert abs(err - r.err) <= 1e-9 * r.err + 1e-12   # FP64 rounding of a unit mass
