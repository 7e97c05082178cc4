"""Host logic of the continuous-batching server (no GPU): admission by budget,
FIFO order, warm-start bookkeeping across ticks, retirement and metrics."""
import math

import numpy as np

from paper_2202_10042_gb300 import serve


class FakeSlot:
    def __init__(self, req):
        self.req = req
        self.done_iters = 0
        self.bytes = serve.device_bytes(req)


def fake_solver(conv_iters):
    """Each request converges after conv_iters[rid] total iterations."""
    calls = []

    def solve(slots, iters):
        calls.append([(s.req.rid, s.done_iters, it) for s, it in zip(slots, iters)])
        out = []
        for s, it in zip(slots, iters):
            need = conv_iters[s.req.rid] - s.done_iters
            if need <= it:
                out.append((1.0 + s.req.rid, 0, max(0, need), 1e-9))
            else:
                out.append((1.0 + s.req.rid, 5, it, 1.0))
        return out
    return solve, calls


def req(rid, n, arrival=0.0, itr_max=1000):
    a = np.full(n, 1.0 / n)
    return serve.Request(rid, a, a.copy(), (1.0 / n,), 0.01, 1e-6, itr_max, arrival)


def test_budget_admission_fifo_and_retire():
    t = [0.0]
    solve, calls = fake_solver({0: 250, 1: 100, 2: 50, 3: 500})
    reqs = [req(0, 1000), req(1, 1000), req(2, 1000), req(3, 1000)]
    one = serve.device_bytes(reqs[0])
    srv = serve.Server(2 * one + 10, tick_iters=100, solve_fn=solve, clock=lambda: t[0], make_slot=FakeSlot)
    for r in reqs:
        srv.submit(r)
    assert srv.admit(0.0) == 2 and [s.req.rid for s in srv.active] == [0, 1]
    t[0] = 1.0
    assert srv.tick(0.0) == 1                     # request 1 converged in the first tick
    assert srv.used == one
    assert srv.admit(1.0) == 1 and [s.req.rid for s in srv.active] == [0, 2]
    assert srv.admitted_while_busy == 1
    while srv.active or srv.waiting:
        t[0] += 1.0
        srv.tick(0.0)
        srv.admit(t[0])
    done = {r.rid: r for r in srv.finished}
    assert sorted(done) == [0, 1, 2, 3]
    assert done[0].iters == 250 and done[0].ticks == 3 and done[0].status == 0
    assert done[3].iters == 500 and done[3].status == 0
    # warm-start bookkeeping: each tick starts where the previous one stopped
    starts = [c for call in calls for c in call if c[0] == 0]
    assert [s[1] for s in starts] == [0, 100, 200]


def test_cap_and_oversize_rejection():
    t = [0.0]
    solve, _ = fake_solver({0: 10**9, 1: 10})
    big = req(1, 10**7)
    srv = serve.Server(serve.device_bytes(req(0, 1000)) + 10, tick_iters=300, solve_fn=solve,
                       clock=lambda: t[0], make_slot=FakeSlot)
    srv.submit(req(0, 1000, itr_max=700))
    srv.submit(big)
    srv.admit(0.0)
    assert big.status == 2 and big in srv.finished
    for _ in range(5):
        t[0] += 1
        srv.tick(0.0)
    r0 = [r for r in srv.finished if r.rid == 0][0]
    assert r0.status == 5 and r0.iters == 700


def test_summary_percentiles():
    rs = []
    for i in range(100):
        r = req(i, 10, arrival=0.0)
        r.finish = float(i + 1)
        r.status = 0
        r.iters = 10
        rs.append(r)
    s = serve.summarize(rs, 100.0)
    assert s["p50_s"] == 50.0 and s["p99_s"] == 99.0 and s["completed"] == 100
    assert math.isclose(s["nit_per_s"], 100 * 10 * 10 / 100.0)


def test_split_by_dim_runs_both_groups_and_keeps_order():
    """The tick's 1D and 2D requests go to their own solve functions (run
    concurrently) and the results come back in slot order."""
    import concurrent.futures as cf
    import threading

    seen = {}

    def make(tag):
        def solve(slots, iters):
            seen[tag] = ([s.req.rid for s in slots], list(iters), threading.get_ident())
            return [(float(s.req.rid), 0, it, 0.0) for s, it in zip(slots, iters)]
        return solve

    slots = []
    for rid, nd in enumerate([1, 2, 1, 2, 2]):
        a = np.full((4,) * nd, 1.0 / 4 ** nd)
        slots.append(FakeSlot(serve.Request(rid, a, a.copy(), (0.25,) * nd, 0.1, 1e-6, 10)))
    with cf.ThreadPoolExecutor(max_workers=2) as pool:
        fn = serve.split_by_dim(make("1d"), make("2d"), pool)
        out = fn(slots, [5, 6, 7, 8, 9])
    assert seen["1d"][:2] == ([0, 2], [5, 7])
    assert seen["2d"][:2] == ([1, 3, 4], [6, 8, 9])
    assert [o[0] for o in out] == [0.0, 1.0, 2.0, 3.0, 4.0]
    assert [o[2] for o in out] == [5, 6, 7, 8, 9]
