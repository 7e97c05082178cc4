"""The allocation-free entry point fs1_w1_noalloc, for callers that cannot call
cudaMalloc (a memory manager that already owns the device's memory, an
embedding that forbids the library from holding device memory), agrees with
fs1_w1 on the same problem, on two calls in a row: the second call finds the
first call's contents in the shared static scratch.  Both run the same team
kernel on the same team size and inputs, so the results are bit-identical.

Kept in its own file, collected last."""
import math

import numpy as np
import pytest

from paper_2202_10042_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2202_10042_gb300 import fs1
    fs1.load()
    return torch, fs1


def _same(x, y):
    return (math.isnan(x) and math.isnan(y)) or x == y


@pytest.mark.parametrize("variant,prec,n,eps,itr,dtype", [
    ("log", "fp32", 131072 + 13, 2e-4, 150, "f64"),   # several CTAs: exchange slots in use
    ("log", "fp32", 131072 + 13, 2e-4, 150, "f32"),   # FP32 inputs
    ("log", "fp32", 1000, 1e-2, 300, "f64"),
    ("plain", "fp64", 1000, 1e-2, 300, "f64"),
])
def test_noalloc_matches_w1_twice(env, variant, prec, n, eps, itr, dtype):
    torch, fs1 = env
    p = inputs.workload2(5, n=n, eps=eps, itr_max=itr)
    td = torch.float32 if dtype == "f32" else torch.float64
    a = torch.tensor(p.a, dtype=td, device="cuda")
    b = torch.tensor(p.b, dtype=td, device="cuda")
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
        assert info2.team_size == info_ref.team_size
        assert info2.iters == info_ref.iters
        assert _same(w2, w_ref), (w2, w_ref)
        assert _same(info2.marginal_err, info_ref.marginal_err)


def test_noalloc_rejects_bad_inputs(env):
    torch, fs1 = env
    p = inputs.workload1(0, itr_max=10)
    a = torch.tensor(p.a, dtype=torch.float64, device="cuda")
    b = torch.tensor(p.b, dtype=torch.float64, device="cuda")
    cfg = fs1.fs1_config_default()
    # an explicit team beyond the co-resident limit
    cfg.team_size = 10000
    st, w, info = fs1.fs1_w1_noalloc(cfg, fs1.Solver.problem(a, b, p.h[0], p.eps, p.tol, p.itr_max))
    assert st == fs1.FS1_EINVAL
    # host memory is not staged on this path
    ha, hb = a.cpu(), b.cpu()
    st, w, info = fs1.fs1_w1_noalloc(None, fs1.Solver.problem(ha, hb, p.h[0], p.eps, p.tol, p.itr_max))
    assert st == fs1.FS1_EINVAL
    # unequal masses
    b2 = b * 1.01
    st, w, info = fs1.fs1_w1_noalloc(None, fs1.Solver.problem(a, b2, p.h[0], p.eps, p.tol, p.itr_max))
    assert st == fs1.FS1_EINVAL and math.isnan(w)
    # a negative entry (masses still equal)
    a3 = a.clone()
    a3[3] = -a3[3]
    a3[4] += 2 * a[3]
    st, w, info = fs1.fs1_w1_noalloc(None, fs1.Solver.problem(a3, b, p.h[0], p.eps, p.tol, p.itr_max))
    assert st == fs1.FS1_EINVAL
    # a valid call after the rejections still agrees with fs1_w1
    prob = fs1.Solver.problem(a, b, p.h[0], p.eps, p.tol, p.itr_max)
    s = fs1.Solver("log", "fp32", autotune=False)
    st_ref, w_ref, _ = fs1.fs1_w1(s.h, prob)
    s.close()
    st, w, _ = fs1.fs1_w1_noalloc(None, prob)
    assert st == st_ref and _same(w, w_ref)
