"""The paper's own synthetic experiments (Section 5.1-5.3) on the GPU, against
the FP64 oracle at the same iteration counts."""
import math

import numpy as np
import pytest

from oracle import cref
from paper_2202_10042_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL64 = 1e-6
TOL32 = 1e-4


@pytest.fixture(scope="module")
def env():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2202_10042_gb300 import fs1
    fs1.load()
    return torch, fs1


def _solve(env, variant, prec, ps, itr=None):
    torch, fs1 = env
    s = fs1.Solver(variant, prec)
    dt = torch.float64 if prec == "fp64" else torch.float32
    keep, probs = [], []
    for p in ps:
        a = torch.tensor(p.a, dtype=dt, device="cuda")
        b = torch.tensor(p.b, dtype=dt, device="cuda")
        keep += [a, b]
        h = tuple(p.h) if p.ndim == 2 else p.h[0]
        probs.append(fs1.Solver.problem(a, b, h, p.eps, p.tol, itr if itr is not None else p.itr_max))
    st, w, infos = s.solve(probs)
    s.close()
    return w, infos


def _ref(p, iters, tau):
    h = tuple(p.h) if p.ndim == 2 else p.h[0]
    return cref.solve(p.a, p.b, h, p.eps, 0.0, iters, tau=tau)


@pytest.mark.parametrize("n", [500, 2000])
def test_e1_random_1d(env, n):
    """Section 5.1: U[0, 1] histograms on [-3, 3], eps = 1e-3, 1000 iterations."""
    _, fs1 = env
    ps = [inputs.paper_e1(i, n=n) for i in range(3)]
    for variant, prec, tol in (("log", "fp32", TOL32), ("plain", "fp64", TOL64)):
        w, infos = _solve(env, variant, prec, ps)
        for k, p in enumerate(ps):
            assert infos[k].iters == 1000 and infos[k].status == fs1.FS1_ENOTCONV
            r = _ref(p, 1000, 1e10)
            assert abs(w[k] - r.w) <= tol * abs(r.w), (variant, n, k, w[k], r.w)
            assert abs(infos[k].marginal_err - r.err) <= 1e-3 * r.err


def test_e2_ricker(env):
    """Section 5.2: the Ricker pair, eps = 1e-2, 500 iterations."""
    _, fs1 = env
    p = inputs.paper_e2(0, n=2000)
    r = _ref(p, 500, 1e10)
    for variant, prec, tol in (("log", "fp32", TOL32), ("plain", "fp64", TOL64)):
        w, infos = _solve(env, variant, prec, [p])
        assert infos[0].iters == 500
        assert abs(w[0] - r.w) <= tol * abs(r.w), (variant, w[0], r.w)


def test_e2_plain_terminates_abnormally_stabilised_does_not(env):
    """Section 5.2 (Fig. 2 right): at small eps the unstabilised iteration
    overflows and stops abnormally; the stabilised one runs on.  With the
    Section 5.1 grid the FP64 plain form overflows at N = 2000, eps = 5e-4."""
    _, fs1 = env
    p = inputs.paper_e2(0, n=2000, eps=5e-4)
    rp = _ref(p, 500, math.inf)
    assert rp.iters < 500 and math.isnan(rp.w)          # the oracle's plain form stops abnormally
    w, infos = _solve(env, "plain", "fp64", [p])
    assert infos[0].status == fs1.FS1_ENUMERIC
    assert abs(infos[0].iters - rp.iters) <= 1
    rs = _ref(p, 500, 1e10)
    w, infos = _solve(env, "log", "fp32", [p])
    assert infos[0].status == fs1.FS1_ENOTCONV and infos[0].iters == 500 and math.isfinite(w[0])
    assert abs(w[0] - rs.w) <= TOL32 * abs(rs.w), (w[0], rs.w)


@pytest.mark.parametrize("side", [20, 40])
def test_e3_random_2d(env, side):
    """Section 5.3: N x N U[0, 1] values, h = 1, eps = 1e-2 (lam = e^-100),
    1000 iterations; the 2D kernel takes its extended-range line scan."""
    _, fs1 = env
    ps = [inputs.paper_e3(i, side=side) for i in range(2)]
    w, infos = _solve(env, "log", "fp32", ps)
    for k, p in enumerate(ps):
        r = _ref(p, 1000, 1e10)
        assert infos[k].iters == 1000
        assert abs(w[k] - r.w) <= TOL32 * abs(r.w), (side, k, w[k], r.w)
