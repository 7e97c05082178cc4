"""The allocation-free entry point fs1_w1_noalloc, for callers that cannot call
cudaMalloc, agrees with fs1_w1 on the same problem, on two calls in a row (the
second call finds the first call's contents in the shared static scratch).

Kept in its own file, collected last."""
import math

import numpy as np
import pytest

from paper_2202_10042_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL32 = 1e-4
TOL64 = 1e-6


@pytest.fixture(scope="module")
def env():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2202_10042_gb300 import fs1
    fs1.load()
    return torch, fs1


@pytest.mark.parametrize("variant,prec,n,eps,itr,tol", [
    ("log", "fp32", 131072 + 13, 2e-4, 150, TOL32),   # several CTAs: exchange slots in use
    ("log", "fp32", 1000, 1e-2, 300, TOL32),
    ("plain", "fp64", 1000, 1e-2, 300, TOL64),
])
def test_noalloc_matches_w1_twice(env, variant, prec, n, eps, itr, tol):
    torch, fs1 = env
    p = inputs.workload2(5, n=n, eps=eps, itr_max=itr)
    a = torch.tensor(p.a, dtype=torch.float64, device="cuda")
    b = torch.tensor(p.b, dtype=torch.float64, device="cuda")
    prob = fs1.Solver.problem(a, b, p.h[0], p.eps, p.tol, p.itr_max)
    # the allocation-free path has no handle and so no autotuner table: compare
    # with fs1_w1 at the same (heuristic) team size
    s = fs1.Solver(variant, prec, autotune=False)
    st, w_ref, info_ref = fs1.fs1_w1(s.h, prob)
    cfg = s.cfg
    s.close()
    assert st in (fs1.FS1_OK, fs1.FS1_ENOTCONV)
    for _ in range(2):
        st2, w2, info2 = fs1.fs1_w1_noalloc(cfg, prob)
        assert st2 == st
        assert info2.iters == info_ref.iters
        assert abs(w2 - w_ref) <= tol * abs(w_ref)
        assert abs(info2.marginal_err - info_ref.marginal_err) <= tol * abs(info_ref.marginal_err)


def test_noalloc_rejects_oversized_team_and_host_memory(env):
    torch, fs1 = env
    p = inputs.workload1(0, itr_max=10)
    a = torch.tensor(p.a, dtype=torch.float64, device="cuda")
    b = torch.tensor(p.b, dtype=torch.float64, device="cuda")
    cfg = fs1.fs1_config_default()
    cfg.team_size = 10000
    st, w, info = fs1.fs1_w1_noalloc(cfg, fs1.Solver.problem(a, b, p.h[0], p.eps, p.tol, p.itr_max))
    assert st == fs1.FS1_EINVAL
    ha, hb = a.cpu(), b.cpu()
    st, w, info = fs1.fs1_w1_noalloc(None, fs1.Solver.problem(ha, hb, p.h[0], p.eps, p.tol, p.itr_max))
    assert st == fs1.FS1_EINVAL
