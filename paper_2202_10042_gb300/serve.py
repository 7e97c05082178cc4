"""Continuous-batching server for FS-1 solves on one GPU.

Requests (1D or 2D histograms with their h, eps, tol and iteration cap) arrive
over time.  The server keeps every admitted request's state on the device (its
a, b and log potentials f, g) and runs *ticks*: one fs1_solve_batch call over
all admitted requests for at most `tick_iters` iterations, warm-started from
the potentials the previous tick left (the solver resumes a pair exactly where
it stopped).  After each tick, converged requests (marginal error <= tol) and
requests that used their iteration cap retire and free their memory; requests
that arrived meanwhile are admitted, first come first served, while the HBM
budget allows, and join the next tick.  Work of all admitted requests of a
tick runs in the same persistent launches (1D pairs of all sizes share one
launch; 2D images share one), so new arrivals overlap with running solves
instead of waiting for them; the 1D and the 2D launches of a tick are issued
concurrently on two CUDA streams (two library handles), with one join per
tick.

The baseline `serve_one_at_a_time` solves each request alone with one call,
in arrival order.

Only argument marshalling and bookkeeping happen here; every iteration runs in
the CUDA library.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import math
import statistics
import time
from collections import deque
from typing import Callable, List, Optional, Sequence

import numpy as np


@dataclasses.dataclass
class Request:
    rid: int
    a: np.ndarray            # (n,) or (n_slow, n_fast)
    b: np.ndarray
    h: tuple
    eps: float
    tol: float
    itr_max: int
    arrival: float = 0.0     # seconds from the start of the run
    # results
    admit: float = math.nan
    finish: float = math.nan
    w1: float = math.nan
    iters: int = 0
    err: float = math.nan
    status: int = -1
    ticks: int = 0

    @property
    def npoints(self) -> int:
        return int(self.a.size)

    @property
    def latency(self) -> float:
        return self.finish - self.arrival


def device_bytes(req: Request) -> int:
    """Device memory a request holds while admitted: a, b (FP32), f, g (FP64)
    and the solver workspace of its launch (2D and 3D keep 40 B per point)."""
    n = req.npoints
    return n * (4 + 4 + 8 + 8) + (40 * n if req.a.ndim >= 2 else 0) + 4096


class _Slot:
    """Device-resident state of an admitted request."""

    def __init__(self, req: Request, torch, device):
        self.req = req
        self.a = torch.as_tensor(np.ascontiguousarray(req.a, dtype=np.float32), device=device)
        self.b = torch.as_tensor(np.ascontiguousarray(req.b, dtype=np.float32), device=device)
        self.f = torch.empty(req.a.shape, dtype=torch.float64, device=device)
        self.g = torch.empty(req.a.shape, dtype=torch.float64, device=device)
        self.done_iters = 0
        self.bytes = device_bytes(req)


def library_solver(solver):
    """solve_fn(slots, iters_each) for the CUDA library: one batched call."""
    from . import fs1

    def solve(slots: Sequence[_Slot], iters: Sequence[int]):
        probs = []
        for s, it in zip(slots, iters):
            warm = s.done_iters > 0
            probs.append(fs1.Solver.problem(s.a, s.b, s.req.h if s.req.a.ndim >= 2 else s.req.h[0],
                                            s.req.eps, s.req.tol, it,
                                            f_out=s.f, g_out=s.g,
                                            f_init=s.f if warm else None,
                                            g_init=s.g if warm else None))
        st, w, infos = solver.solve(probs)
        return [(float(w[k]), int(i.status), int(i.iters), float(i.marginal_err)) for k, i in enumerate(infos)]
    return solve


def split_by_dim(solve_1d: Callable, solve_2d: Callable, pool) -> Callable:
    """solve_fn that runs a tick's 1D and 2D requests as two concurrent calls
    (two library handles on two CUDA streams, each call ending in its own
    stream synchronisation), so their device work overlaps; the results come
    back in slot order."""

    def solve(slots: Sequence, iters: Sequence[int]):
        one = [k for k, s in enumerate(slots) if s.req.a.ndim == 1]
        two = [k for k, s in enumerate(slots) if s.req.a.ndim != 1]
        jobs = []
        for idx, fn in ((one, solve_1d), (two, solve_2d)):
            if idx:
                jobs.append((idx, pool.submit(fn, [slots[k] for k in idx], [iters[k] for k in idx])))
        out = [None] * len(slots)
        for idx, fut in jobs:
            for k, r in zip(idx, fut.result()):
                out[k] = r
        return out
    return solve


class Server:
    """Admission by HBM budget, ticks of `tick_iters` iterations, retire on
    convergence or cap.  `solve_fn(slots, iters)` returns per slot
    (w1, status, iters_done_in_tick, marginal_err)."""

    OK, ENOTCONV = 0, 5

    def __init__(self, budget_bytes: int, tick_iters: int = 200, solve_fn: Optional[Callable] = None,
                 device="cuda", clock: Callable[[], float] = time.perf_counter, make_slot=None):
        self.budget = int(budget_bytes)
        self.tick_iters = int(tick_iters)
        self.used = 0
        self.waiting: deque = deque()
        self.active: List[_Slot] = []
        self.finished: List[Request] = []
        self.clock = clock
        self.ticks = 0
        self.admitted_while_busy = 0
        self._make_slot = make_slot
        self._solvers = []
        self._pool = None
        if solve_fn is None:
            import concurrent.futures as cf
            import torch
            from . import fs1
            self._torch = torch
            self._device = device
            # 1D and 2D requests on their own handle and stream, solved concurrently
            self._streams = [torch.cuda.Stream(device=device) for _ in range(2)]
            self._solvers = [fs1.Solver("log", "fp32", stream=st.cuda_stream) for st in self._streams]
            self._pool = cf.ThreadPoolExecutor(max_workers=2)
            solve_fn = split_by_dim(library_solver(self._solvers[0]), library_solver(self._solvers[1]), self._pool)
        self.solve_fn = solve_fn

    def close(self):
        for s in self._solvers:
            s.close()
        self._solvers = []
        if self._pool is not None:
            self._pool.shutdown()
            self._pool = None

    # -- admission ---------------------------------------------------------
    def submit(self, req: Request):
        self.waiting.append(req)

    def admit(self, now: float) -> int:
        n = 0
        busy = bool(self.active)   # requests already running when these arrive
        while self.waiting:
            req = self.waiting[0]
            need = device_bytes(req)
            if need > self.budget:
                # can never fit: reject
                self.waiting.popleft()
                req.status = 2   # FS1_ENOMEM
                req.admit = req.finish = now
                self.finished.append(req)
                continue
            if self.used + need > self.budget:
                break
            self.waiting.popleft()
            slot = self._make_slot(req) if self._make_slot else _Slot(req, self._torch, self._device)
            req.admit = now
            if busy:
                self.admitted_while_busy += 1
            self.active.append(slot)
            self.used += slot.bytes
            n += 1
        if n and self._make_slot is None:
            # the new requests' uploads (on torch's stream) complete before the
            # solver streams read them
            self._torch.cuda.current_stream(self._device).synchronize()
        return n

    # -- one tick ----------------------------------------------------------
    def tick(self, t0: float):
        if not self.active:
            return 0
        iters = [min(self.tick_iters, s.req.itr_max - s.done_iters) for s in self.active]
        res = self.solve_fn(self.active, iters)
        self.ticks += 1
        now = self.clock() - t0
        keep = []
        retired = 0
        for s, (w, st, it, err) in zip(self.active, res):
            s.done_iters += it
            s.req.ticks += 1
            r = s.req
            r.w1, r.err, r.iters = w, err, s.done_iters
            # an unconverged request that made no progress in its tick (only a
            # failed solve does that) retires instead of looping
            if st == self.ENOTCONV and s.done_iters < r.itr_max and it > 0:
                keep.append(s)
                continue
            r.status = st
            r.finish = now
            self.finished.append(r)
            self.used -= s.bytes
            retired += 1
        self.active = keep
        return retired

    # -- real-time run -----------------------------------------------------
    def run(self, requests: Sequence[Request], max_seconds: float = math.inf) -> dict:
        pending = deque(sorted(requests, key=lambda r: r.arrival))
        t0 = self.clock()
        while pending or self.waiting or self.active:
            now = self.clock() - t0
            if now > max_seconds:
                break
            while pending and pending[0].arrival <= now:
                self.submit(pending.popleft())
            self.admit(now)
            if not self.active:
                if pending:
                    time.sleep(max(0.0, min(0.01, pending[0].arrival - now)))
                continue
            self.tick(t0)
        return summarize(self.finished, self.clock() - t0)


def summarize(done: Sequence[Request], makespan: float) -> dict:
    ok = [r for r in done if r.status in (0, 5)]
    lat = sorted(r.latency for r in ok)
    nit = sum(r.npoints * r.iters for r in ok)

    def pct(p):
        if not lat:
            return math.nan
        k = min(len(lat) - 1, max(0, int(math.ceil(p / 100.0 * len(lat))) - 1))
        return lat[k]
    return {"requests": len(done), "completed": len(ok), "makespan_s": makespan,
            "throughput_rps": len(ok) / makespan if makespan > 0 else math.nan,
            "nit_per_s": nit / makespan if makespan > 0 else math.nan,
            "p50_s": pct(50), "p99_s": pct(99),
            "converged": sum(1 for r in ok if r.status == 0)}


def serve_one_at_a_time(requests: Sequence[Request], solver=None, clock=time.perf_counter,
                        max_seconds: float = math.inf) -> dict:
    """Baseline: each request alone in one call, first come first served."""
    import torch
    from . import fs1
    own = solver is None
    solver = solver or fs1.Solver("log", "fp32")
    done = []
    t0 = clock()
    for r in sorted(requests, key=lambda r: r.arrival):
        now = clock() - t0
        if now > max_seconds:
            break
        if r.arrival > now:
            time.sleep(r.arrival - now)
        a = torch.as_tensor(np.ascontiguousarray(r.a, dtype=np.float32), device="cuda")
        b = torch.as_tensor(np.ascontiguousarray(r.b, dtype=np.float32), device="cuda")
        st, w, info = fs1.fs1_w1(solver.h, fs1.Solver.problem(a, b, r.h if r.a.ndim >= 2 else r.h[0], r.eps,
                                                              r.tol, r.itr_max))
        r.admit = r.arrival
        r.finish = clock() - t0
        r.w1, r.status, r.iters, r.err = w, info.status, info.iters, info.marginal_err
        done.append(r)
    if own:
        solver.close()
    return summarize(done, clock() - t0)


def make_requests(rate: float, duration: float, **kw) -> List[Request]:
    """Requests of the serving workload (seeded Poisson arrivals)."""
    from . import inputs
    arr = inputs.workload5_arrivals(rate, duration)
    out = []
    for i, t in enumerate(arr):
        p = inputs.workload5(i, arrival=float(t), **kw)
        out.append(Request(i, p.a, p.b, tuple(p.h), p.eps, p.tol, p.itr_max, float(t)))
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description="FS-1 serving benchmark (continuous batching vs one-at-a-time)")
    ap.add_argument("--rate", type=float, default=2000.0)
    ap.add_argument("--duration", type=float, default=60.0)
    ap.add_argument("--budget-gb", type=float, default=40.0)
    ap.add_argument("--tick-iters", type=int, default=200)
    ap.add_argument("--max-seconds", type=float, default=120.0)
    ap.add_argument("--n-max", type=int, default=1000000)
    ap.add_argument("--side-max", type=int, default=1024)
    ap.add_argument("--baseline", action="store_true")
    args = ap.parse_args(argv)
    reqs = make_requests(args.rate, args.duration, n_range=(1000, args.n_max), side_range=(64, args.side_max))
    srv = Server(int(args.budget_gb * 1e9), args.tick_iters)
    s = srv.run(reqs, args.max_seconds)
    s.update({"mode": "continuous", "offered_rps": args.rate, "ticks": srv.ticks,
              "admitted_while_busy": srv.admitted_while_busy})
    srv.close()
    print(json.dumps(s))
    if args.baseline:
        reqs = make_requests(args.rate, args.duration, n_range=(1000, args.n_max), side_range=(64, args.side_max))
        b = serve_one_at_a_time(reqs, max_seconds=args.max_seconds)
        b.update({"mode": "one_at_a_time", "offered_rps": args.rate})
        print(json.dumps(b))


if __name__ == "__main__":
    main()
