"""Graph replay of the 1D batch call, the device-side input check, and the
team-size autotuner with its cache file."""
import math
import types

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


def _pair(n, index, h, eps, tol, itr_max):
    a, b = inputs.random_pair_1d(index, n)
    return types.SimpleNamespace(a=a, b=b, h=(h,), eps=eps, tol=tol, itr_max=itr_max)


def _tensors(torch, ps):
    out = []
    for p in ps:
        out.append((torch.tensor(p.a, dtype=torch.float32, device="cuda"),
                    torch.tensor(p.b, dtype=torch.float32, device="cuda")))
    return out


def _probs(fs1, ps, ts, itr=None):
    return [fs1.Solver.problem(a, b, p.h[0], p.eps, p.tol, itr if itr is not None else p.itr_max)
            for p, (a, b) in zip(ps, ts)]


def test_graph_replay_matches_direct_launches(env):
    torch, fs1 = env
    ps = [inputs.workload3(i, itr_max=120, n_range=(2000, 40000)) for i in range(10)]
    ts = _tensors(torch, ps)
    probs = _probs(fs1, ps, ts)
    direct = fs1.Solver("log", "fp32", autotune=False, use_graph=False)
    _, w_ref, i_ref = direct.solve(probs)
    assert direct.stats()["graphs_captured"] == 0
    direct.close()
    s = fs1.Solver("log", "fp32", autotune=False)
    runs = []
    for _ in range(4):
        l0 = fs1.fs1_launch_count()
        st, w, infos = s.solve(probs)
        assert fs1.fs1_launch_count() - l0 == 2      # input check + team kernel
        runs.append((w, infos))
    stats = s.stats()
    # call 1 direct, call 2 captures and launches the graph, calls 3-4 replay it
    assert stats["graphs_captured"] == 1 and stats["graph_replays"] == 3
    for w, infos in runs:
        # the same launch (team sizes, plan) is bit-identical
        assert np.array_equal(w, w_ref)
        for a, b in zip(infos, i_ref):
            assert a.iters == b.iters and a.status == b.status and a.marginal_err == b.marginal_err
            assert math.isfinite(a.ms) and a.ms > 0.0
    # a replay reads the new header: other inputs of the same shape
    # (same sizes, so the same signature; new histograms)
    ps2 = [_pair(p.a.size, 500 + k, p.h[0], p.eps, p.tol, 120) for k, p in enumerate(ps)]
    ts2 = _tensors(torch, ps2)
    probs2 = _probs(fs1, ps2, ts2)
    _, w2, i2 = s.solve(probs2)
    assert s.stats()["graph_replays"] == 4
    refs = cref.solve_many([(p.a, p.b, p.h[0], p.eps, 0.0, i2[k].iters) for k, p in enumerate(ps2)], tau=1e10)
    for k, r in enumerate(refs):
        assert abs(w2[k] - r.w) <= TOL32 * abs(r.w), (k, w2[k], r.w)
    s.close()


def test_invalid_pair_reported_by_device_check(env):
    torch, fs1 = env
    ps = [inputs.workload3(i, itr_max=80, n_range=(2000, 20000)) for i in range(6)]
    ts = _tensors(torch, ps)
    bad_neg = ts[1][0].clone()
    bad_neg[5] = -1e-3
    bad_mass = ts[4][1] * 1.01
    ts_bad = list(ts)
    ts_bad[1] = (bad_neg, ts[1][1])
    ts_bad[4] = (ts[4][0], bad_mass)
    s = fs1.Solver("log", "fp32", autotune=False)
    _, w_ok, i_ok = s.solve(_probs(fs1, ps, ts))
    for _ in range(3):   # direct, captured, replayed
        st, w, infos = s.solve(_probs(fs1, ps, ts_bad))
        assert st == fs1.FS1_EINVAL
        for k in range(6):
            if k in (1, 4):
                assert infos[k].status == fs1.FS1_EINVAL and math.isnan(w[k])
            else:
                assert infos[k].status == i_ok[k].status and w[k] == w_ok[k]
    s.close()


def test_autotuner_picks_and_caches(env, tmp_path, monkeypatch):
    torch, fs1 = env
    cache = tmp_path / "fs1_tune.txt"
    monkeypatch.setenv("FS1_AUTOTUNE_CACHE", str(cache))
    # one size class: 24 pairs of N = 2^17
    n = 1 << 17
    ps = [_pair(n, 900 + k, 1.0 / n, 0.1, 1e-9, 60) for k in range(24)]
    ts = _tensors(torch, ps)
    probs = _probs(fs1, ps, ts)
    s = fs1.Solver("log", "fp32", trial_iters=8)
    _, w, infos = s.solve(probs)
    st1 = s.stats()
    assert st1["tuned_classes"] == 1 and st1["trial_launches"] >= 1
    s.close()
    lines = cache.read_text().split("\n")
    lines = [ln for ln in lines if ln.strip()]
    assert len(lines) == 1
    key, T = lines[0].split()
    assert int(T) >= 1 and int(T) == infos[0].team_size
    # a new handle reads the table and runs no trials
    s2 = fs1.Solver("log", "fp32")
    _, w2, infos2 = s2.solve(probs)
    st2 = s2.stats()
    assert st2["trial_launches"] == 0 and st2["tuned_classes"] == 1
    assert infos2[0].team_size == int(T)
    assert np.array_equal(w, w2)
    s2.close()
    refs = cref.solve_many([(p.a, p.b, p.h[0], p.eps, 0.0, infos[k].iters) for k, p in enumerate(ps[:4])],
                           tau=1e10)
    for k, r in enumerate(refs):
        assert abs(w[k] - r.w) <= TOL32 * abs(r.w)
