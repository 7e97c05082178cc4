"""Uneven batches in one persistent launch (workload 3 shape): parity against
the CPU FP64 oracle per pair, and the same result alone and in the mix."""
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


def _solve(env, ps, **kw):
    torch, fs1 = env
    s = fs1.Solver("log", "fp32", **kw)
    keep, probs = [], []
    for p in ps:
        a = torch.tensor(p.a, dtype=torch.float64, device="cuda")
        b = torch.tensor(p.b, dtype=torch.float64, device="cuda")
        keep += [a, b]
        probs.append(fs1.Solver.problem(a, b, p.h[0], p.eps, p.tol, p.itr_max))
    st, w, infos = s.solve(probs)
    s.close()
    return w, infos


def test_workload3_sample_against_oracle(env):
    _, fs1 = env
    ps = [inputs.workload3(i, itr_max=150) for i in range(40)]
    w, infos = _solve(env, ps)
    refs = cref.solve_many([(p.a, p.b, p.h[0], p.eps, 0.0, infos[k].iters) for k, p in enumerate(ps)],
                           tau=1e10)
    ns = sorted(p.a.size for p in ps)
    assert ns[0] < 2000 and ns[-1] > 20000   # the sample spans several team classes
    for k, (p, r) in enumerate(zip(ps, refs)):
        assert infos[k].status in (fs1.FS1_OK, fs1.FS1_ENOTCONV)
        assert abs(w[k] - r.w) <= TOL32 * abs(r.w), (k, p.a.size, p.eps, w[k], r.w)
        if infos[k].status == fs1.FS1_OK:
            assert infos[k].marginal_err <= p.tol


def test_same_alone_and_in_mix(env):
    ps = [inputs.workload3(i, itr_max=400) for i in range(24)]
    w_mix, i_mix = _solve(env, ps)
    for k in (0, 7, 13, 23):
        w1, i1 = _solve(env, [ps[k]])
        assert i1[0].iters == i_mix[k].iters or abs(i1[0].iters - i_mix[k].iters) <= 1
        assert abs(w1[0] - w_mix[k]) <= TOL32 * abs(w_mix[k])


def test_forced_team_size_and_order_independence(env):
    ps = [inputs.workload3(i, itr_max=100, n_range=(3000, 30000)) for i in range(12)]
    w_a, _ = _solve(env, ps)
    w_b, _ = _solve(env, ps[::-1])
    w_c, _ = _solve(env, ps, team_size=8)
    for k in range(12):
        assert abs(w_a[k] - w_b[11 - k]) <= TOL32 * abs(w_a[k])
        assert abs(w_a[k] - w_c[k]) <= TOL32 * abs(w_a[k])


def _pair(seed, n, eps, itr):
    rng = np.random.default_rng(seed)
    a = rng.uniform(0.05, 1.0, n)
    b = rng.uniform(0.05, 1.0, n)
    return inputs.Problem(a / a.sum(), b / b.sum(), (1.0 / n,), eps, 0.0, itr, 1, (n,), 0, seed)


def test_level_schedule_team_sizes_and_parity(env):
    """A batch spanning four team classes (1, 2, 4 and 8 CTAs of 16384 points)
    runs as one level schedule: teams of 8 CTAs take the largest pairs first
    and split into teams of 4, 2 and 1 as the queues empty.  Every pair is
    solved by a team of its class, matches the oracle at its iteration count,
    and gives the same result in the mix as alone; a replay of the captured
    graph gives the same bits."""
    torch, fs1 = env
    itr = 200   # about 400 exchanges per pair: the compact slots' 8-bit tags wrap
    sizes = [100000, 70000, 40000, 33000, 20000, 17000] + [500 + 701 * k for k in range(20)] + [16384, 9000]
    ps = [_pair(700 + k, n, 0.02 if k % 2 else 0.005, itr) for k, n in enumerate(sizes)]
    want_T = [1 << max(0, math.ceil(math.log2(math.ceil(p.a.size / 16384)))) for p in ps]
    assert sorted(set(want_T)) == [1, 2, 4, 8]
    keep, probs = [], []
    for p in ps:
        a = torch.tensor(p.a, dtype=torch.float32, device="cuda")
        b = torch.tensor(p.b, dtype=torch.float32, device="cuda")
        keep += [a, b]
        probs.append(fs1.Solver.problem(a, b, p.h[0], p.eps, p.tol, p.itr_max))
    s = fs1.Solver("log", "fp32")
    runs = [s.solve(probs) for _ in range(3)]   # direct, captured, replayed
    st = s.stats()
    s.close()
    assert st["graph_replays"] >= 1
    _, w, infos = runs[0]
    for _, w2, i2 in runs[1:]:
        assert list(w2) == list(w) and [i.iters for i in i2] == [i.iters for i in infos]
    assert [i.team_size for i in infos] == want_T
    refs = cref.solve_many([(p.a, p.b, p.h[0], p.eps, 0.0, infos[k].iters) for k, p in enumerate(ps)], tau=1e10)
    for k, (p, r) in enumerate(zip(ps, refs)):
        assert infos[k].status in (fs1.FS1_OK, fs1.FS1_ENOTCONV)
        assert abs(w[k] - r.w) <= TOL32 * abs(r.w), (k, p.a.size, w[k], r.w)
        assert abs(infos[k].marginal_err - r.err) <= 1e-3 * r.err + 1e-9, (k, infos[k].marginal_err, r.err)
    for k in (0, 3, 10):
        w1, i1 = _solve(env, [ps[k]], team_size=want_T[k], autotune=False)
        assert i1[0].iters == infos[k].iters
        assert abs(w1[0] - w[k]) <= 1e-5 * abs(w[k])


def test_units_small_pairs(env):
    """Small pairs on the kernel's units (a pair per unit of 8, 4 or one warp,
    after the pairs that need whole CTAs; a batch gets units when its small
    pairs outnumber the co-resident CTAs), mixed with team pairs: each
    matches the oracle at its iteration count (all of the first 27, every
    tenth of the rest) and the same pairs solved on whole CTAs (units off)
    within FP32 rounding; the stop rule stops every converging pair within
    one iteration of the oracle's stop."""
    torch, fs1 = env
    sizes = [33, 100, 257, 640, 1024, 1025, 2000, 3000, 4096, 4097, 6000, 30000, 9, 700, 2500]
    epss = [0.05, 0.02, 0.01, 0.005, 0.002]
    ps = [_pair(900 + k, n, epss[k % 5], 300) for k, n in enumerate(sizes)]
    ps += [inputs.workload3(i, tol=1e-5, itr_max=3000, n_range=(256, 4096)) for i in range(12)]
    ps += [inputs.workload3(1000 + i, tol=0.0, itr_max=40, n_range=(256, 8192)) for i in range(200)]
    checked = set(range(27)) | set(range(27, len(ps), 10))

    def run(units):
        keep, probs = [], []
        for p in ps:
            a = torch.tensor(p.a, dtype=torch.float32, device="cuda")
            b = torch.tensor(p.b, dtype=torch.float32, device="cuda")
            keep += [a, b]
            probs.append(fs1.Solver.problem(a, b, p.h[0], p.eps, p.tol, p.itr_max))
        s = fs1.Solver("log", "fp32", units=units)
        out = [s.solve(probs) for _ in range(3)]
        s.close()
        return out

    on = run(True)
    _, w, infos = on[0]
    for _, w2, i2 in on[1:]:
        assert list(w2) == list(w) and [i.iters for i in i2] == [i.iters for i in infos]
    _, w_off, i_off = run(False)[0]
    # units ran: a unit's pair is summed in another order than on a whole CTA
    assert sum(w_off[k] != w[k] for k in range(len(ps))) > 0
    ks = sorted(checked)
    refs = dict(zip(ks, cref.solve_many([(ps[k].a, ps[k].b, ps[k].h[0], ps[k].eps, 0.0, infos[k].iters)
                                         for k in ks], tau=1e10)))
    for k, p in enumerate(ps):
        assert infos[k].status in (fs1.FS1_OK, fs1.FS1_ENOTCONV), (k, infos[k].status)
        assert abs(i_off[k].iters - infos[k].iters) <= 1
        if i_off[k].iters == infos[k].iters:
            assert abs(w_off[k] - w[k]) <= 1e-5 * abs(w[k]), (k, w_off[k], w[k])
        if k not in refs:
            continue
        r = refs[k]
        assert abs(w[k] - r.w) <= TOL32 * abs(r.w), (k, p.a.size, w[k], r.w)
        # FP32 terms: the error of a pair converged below FP32 resolution floors near 1e-8
        assert abs(infos[k].marginal_err - r.err) <= 1e-3 * r.err + 1e-7, (k, infos[k].marginal_err, r.err)
        if p.tol > 0 and infos[k].status == fs1.FS1_OK:
            ro = cref.solve(p.a, p.b, p.h[0], p.eps, p.tol, p.itr_max, tau=1e10)
            assert abs(ro.iters - infos[k].iters) <= 1, (k, ro.iters, infos[k].iters)
    assert infos[sizes.index(30000)].team_size == 2 and all(infos[k].team_size == 1 for k in range(3))
