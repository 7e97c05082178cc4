"""Continuous batching on the GPU: requests that arrive while others run are
admitted into later ticks, and every result equals the result of the same
request solved alone, within the FP32 tolerance (1e-4 relative W1)."""
import numpy as np
import pytest

from paper_2202_10042_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2202_10042_gb300 import fs1, serve
    fs1.load()
    return torch, fs1, serve


def test_mix_equals_alone(env):
    torch, fs1, serve = env
    reqs = []
    for i in range(14):
        p = inputs.workload5(i, arrival=0.02 * i, n_range=(1000, 60000), side_range=(32, 96),
                             eps_range=(3e-3, 2e-2), itr_max=1200)
        reqs.append(serve.Request(i, p.a, p.b, tuple(p.h), p.eps, p.tol, p.itr_max, p.arrival))
    srv = serve.Server(int(4e9), tick_iters=150)
    summ = srv.run(reqs, max_seconds=300.0)
    srv.close()
    assert summ["completed"] == len(reqs)
    assert srv.ticks >= 2 and srv.admitted_while_busy >= 1
    assert any(r.a.ndim == 2 for r in reqs) and any(r.a.ndim == 1 for r in reqs)
    s = fs1.Solver("log", "fp32")
    for r in reqs:
        a = torch.as_tensor(np.ascontiguousarray(r.a, dtype=np.float32), device="cuda")
        b = torch.as_tensor(np.ascontiguousarray(r.b, dtype=np.float32), device="cuda")
        st, w, info = fs1.fs1_w1(s.h, fs1.Solver.problem(a, b, r.h if r.a.ndim == 2 else r.h[0], r.eps, r.tol,
                                                         r.itr_max))
        assert info.status == r.status, (r.rid, info.status, r.status)
        assert abs(info.iters - r.iters) <= 1, (r.rid, info.iters, r.iters)
        assert abs(w - r.w1) <= 1e-4 * abs(w), (r.rid, w, r.w1)
    s.close()
