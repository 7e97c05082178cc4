"""Edge cases of the 1D path and of the batch entry point, against the FP64
oracle: single points, CTA-boundary sizes, no iterations, an already-met
tolerance, the largest pair that fits on chip and the first that does not,
an empty batch, and one batch mixing 1D, 2D, 3D and invalid problems."""
import math

import numpy as np
import pytest

from oracle import cref
from paper_2202_10042_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL32 = 1e-4


@pytest.fixture(scope="module")
def env():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2202_10042_gb300 import fs1
    fs1.load()
    return torch, fs1


def _problems(torch, fs1, items, dtype=None):
    keep, probs = [], []
    for (a, b, h, eps, tol, itr) in items:
        ta = torch.tensor(a, dtype=dtype or torch.float64, device="cuda")
        tb = torch.tensor(b, dtype=dtype or torch.float64, device="cuda")
        keep += [ta, tb]
        probs.append(fs1.Solver.problem(ta, tb, h, eps, tol, itr))
    return keep, probs


@pytest.mark.parametrize("n", [1, 2, 3, 31, 511, 512, 513, 1025])
def test_small_and_boundary_sizes(env, n):
    torch, fs1 = env
    a, b = inputs.random_pair_1d(n, n, floor=0.01)
    keep, probs = _problems(torch, fs1, [(a, b, 1.0 / n, 0.02, 0.0, 50)])
    s = fs1.Solver("log", "fp32")
    st, w, infos = s.solve(probs)
    s.close()
    ref = cref.solve(a, b, 1.0 / n, 0.02, 0.0, 50, tau=1e10)
    assert infos[0].iters == ref.iters
    if n == 1:
        assert w[0] == 0.0 and ref.w == 0.0
    else:
        assert abs(w[0] - ref.w) <= TOL32 * abs(ref.w), (n, w[0], ref.w)
    assert abs(infos[0].marginal_err - ref.err) <= 1e-3 * ref.err + 1e-7


def test_no_iterations_and_met_tolerance(env):
    """itr_max = 0 returns the initial 1/N iterate; a tolerance the initial
    iterate meets stops at once (reading: the while test precedes the first
    update)."""
    torch, fs1 = env
    n = 700
    a, b = inputs.random_pair_1d(3, n, floor=0.01)
    keep, probs = _problems(torch, fs1, [(a, b, 1 / n, 0.05, 0.0, 0), (a, b, 1 / n, 0.05, 10.0, 100)])
    for variant, prec in (("log", "fp32"), ("plain", "fp64"), ("paper", "fp64")):
        s = fs1.Solver(variant, prec)
        st, w, infos = s.solve(probs)
        s.close()
        for k, (tol, itr) in enumerate(((0.0, 0), (10.0, 100))):
            ref = cref.solve(a, b, 1 / n, 0.05, tol, itr, tau=1e10)
            assert infos[k].iters == ref.iters == 0
            assert abs(w[k] - ref.w) <= TOL32 * abs(ref.w), (variant, k, w[k], ref.w)
        assert infos[1].status == fs1.FS1_OK


def test_largest_pair_on_chip_and_beyond(env):
    """152 CTAs x 512 threads x 32 points = 2490368 points is the largest pair
    the team kernel holds on chip (small c); one team of every SM runs it.  A
    larger pair streams through device memory."""
    torch, fs1 = env
    n = 152 * 512 * 32
    a, b = inputs.random_pair_1d(5, n, floor=0.05)
    eps = 50.0 / n   # c = h / eps = 0.02: 32 points per thread are allowed
    keep, probs = _problems(torch, fs1, [(a, b, 1.0 / n, eps, 0.0, 6)], dtype=torch.float32)
    s = fs1.Solver("log", "fp32", autotune=False)
    st, w, infos = s.solve(probs)
    assert infos[0].status == fs1.FS1_ENOTCONV and infos[0].team_size == 152
    ref = cref.solve(a.astype(np.float32).astype(np.float64), b.astype(np.float32).astype(np.float64),
                     1.0 / n, eps, 0.0, 6, tau=1e10)
    assert abs(w[0] - ref.w) <= TOL32 * abs(ref.w)
    # one CTA more than fits: the stabilised variant streams it through device
    # memory (team size 0); the plain FP32 variant reports FS1_EUNSUPPORTED
    a2, b2 = inputs.random_pair_1d(6, n + 512 * 32, floor=0.05)
    keep2, probs2 = _problems(torch, fs1, [(a2, b2, 1.0 / a2.size, 50.0 / a2.size, 0.0, 6)], dtype=torch.float32)
    st, w, infos = s.solve(probs2)
    s.close()
    assert infos[0].status == fs1.FS1_ENOTCONV and infos[0].team_size == 0
    ref2 = cref.solve(a2.astype(np.float32).astype(np.float64), b2.astype(np.float32).astype(np.float64),
                      1.0 / a2.size, 50.0 / a2.size, 0.0, 6, tau=1e10)
    assert abs(w[0] - ref2.w) <= TOL32 * abs(ref2.w)
    sp = fs1.Solver("plain", "fp32", autotune=False)
    st, w, infos = sp.solve(probs2)
    sp.close()
    assert infos[0].status == fs1.FS1_EUNSUPPORTED


def test_empty_batch(env):
    torch, fs1 = env
    s = fs1.Solver("log", "fp32")
    st, w, infos = s.solve([])
    s.close()
    assert st == fs1.FS1_OK and len(w) == 0 and infos == []


def test_mixed_dimensions_and_invalid_in_one_batch(env):
    torch, fs1 = env
    rng = np.random.default_rng(8)
    items = []
    a1, b1 = inputs.random_pair_1d(9, 3000, floor=0.01)
    items.append((a1, b1, 1 / 3000, 0.01, 0.0, 40))
    a2 = rng.uniform(0.1, 1, (30, 40)); a2 /= a2.sum()
    b2 = rng.uniform(0.1, 1, (30, 40)); b2 /= b2.sum()
    items.append((a2, b2, (1 / 40, 1 / 30), 0.02, 0.0, 40))
    a3 = rng.uniform(0.1, 1, (6, 7, 8)); a3 /= a3.sum()
    b3 = rng.uniform(0.1, 1, (6, 7, 8)); b3 /= b3.sum()
    items.append((a3, b3, (1 / 8, 1 / 7, 1 / 6), 0.05, 0.0, 40))
    bad = b1 * 1.5   # mass mismatch
    items.append((a1, bad, 1 / 3000, 0.01, 0.0, 40))
    keep, probs = _problems(torch, fs1, items)
    s = fs1.Solver("log", "fp32")
    st, w, infos = s.solve(probs)
    s.close()
    assert st == fs1.FS1_EINVAL
    assert infos[3].status == fs1.FS1_EINVAL
    for k in range(3):
        a, b, h, eps, tol, itr = items[k]
        ref = cref.solve(a, b, h, eps, 0.0, itr, tau=1e10)
        assert infos[k].status == fs1.FS1_ENOTCONV and infos[k].iters == itr
        assert abs(w[k] - ref.w) <= TOL32 * abs(ref.w), (k, w[k], ref.w)


def test_bounded_wait_gives_up_without_fault(env):
    """A pair launched as a team of two CTAs of which only one runs: the
    waits for the missing partner's exchange slot end at the spin cap, the
    pair reports FS1_ETIMEOUT, and the handle then solves normally."""
    torch, fs1 = env
    n = 4000
    a, b = inputs.random_pair_1d(11, n, floor=0.05)
    ta = torch.tensor(a, dtype=torch.float64, device="cuda")
    tb = torch.tensor(b, dtype=torch.float64, device="cuda")
    s = fs1.Solver("log", "fp32", autotune=False)
    st, pair_st = fs1.fs1_test_missing_partner(s.h, ta.data_ptr(), tb.data_ptr(), n, 1.0 / n, 0.05, 1 << 14)
    assert st == fs1.FS1_OK and pair_st == fs1.FS1_ETIMEOUT
    st2, w, infos = s.solve([fs1.Solver.problem(ta, tb, 1.0 / n, 0.05, 0.0, 20)])
    s.close()
    assert infos[0].status == fs1.FS1_ENOTCONV and infos[0].iters == 20
    ref = cref.solve(a, b, 1.0 / n, 0.05, 0.0, 20, tau=1e10)
    assert abs(w[0] - ref.w) <= TOL32 * abs(ref.w)
