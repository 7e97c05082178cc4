"""Exact and generic instantiations of the 1D team kernel against the oracle.

A pair of N points on a team of T CTAs gives every thread E = ceil(N / (512 T))
points.  A launch whose pairs share one E runs the exact instantiation of
that E (stabilised FP32: E = 1 .. 32, plain FP64: E = 1 .. 8); other launches
run the generic kernel, whose loops go in chunks of 4 points with identity
steps past E.  Every exact kernel is run here once, each at a ragged N, and
compared with the FP64 oracle at the GPU's iteration count (relative W1
tolerance 1e-4 for FP32, 1e-6 for FP64).
"""
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


def _n_for(E, k=0):
    """A ragged N with ceil(N / 512) = E."""
    return 512 * (E - 1) + 1 + (97 * E + 211 * k) % 512


def _run(env, variant, prec, pairs, team_size, itr):
    torch, fs1 = env
    dt = torch.float64 if prec == "fp64" else torch.float32
    keep, probs = [], []
    for a, b, h, eps in pairs:
        ta = torch.tensor(a, dtype=dt, device="cuda")
        tb = torch.tensor(b, dtype=dt, device="cuda")
        keep += [ta, tb]
        probs.append(fs1.Solver.problem(ta, tb, h, eps, 0.0, itr))
    s = fs1.Solver(variant, prec, team_size=team_size, autotune=False)
    st, w, infos = s.solve(probs)
    stats = s.stats()
    s.close()
    return st, w, infos, stats


def _pairs(ns, cs, seed, floor):
    """Pairs on [0, 1] (h = 1 / N) with eps = h / c: c = h / eps is the decay
    exponent per grid step, lam = e^{-c}."""
    out = []
    for k, n in enumerate(ns):
        a, b = inputs.random_pair_1d(seed + k, n, floor=floor)
        c = cs[k % len(cs)]
        out.append((a, b, 1.0 / n, 1.0 / (c * n)))
    return out


def _check(pairs, w, infos, itr, tau, tol):
    refs = cref.solve_many([(a, b, h, eps, 0.0, itr) for a, b, h, eps in pairs], tau=tau)
    for k, r in enumerate(refs):
        # the FP64 oracle stops early only at an exactly zero marginal error:
        # a fixed point, where further iterations change nothing
        assert infos[k].iters == itr and (r.iters == itr or r.err == 0.0)
        assert abs(w[k] - r.w) <= tol * abs(r.w), (k, w[k], r.w)


@pytest.mark.parametrize("E", list(range(1, 33)))
def test_exact_log_kernel(env, E):
    itr = 40
    # three pairs of the same E: three one-CTA teams in one exact launch
    pairs = _pairs([_n_for(E, k) for k in range(3)], (0.3, 0.05, 0.01), 7000 + 10 * E, 1e-3)
    st, w, infos, stats = _run(env, "log", "fp32", pairs, 1, itr)
    assert stats["last_exact_E"] == E and stats["exact_launches"] == 1
    _check(pairs, w, infos, itr, 1e10, TOL32)


@pytest.mark.parametrize("E", list(range(1, 9)))
def test_exact_plain_fp64_kernel(env, E):
    itr = 40
    pairs = _pairs([_n_for(E, k) for k in range(2)], (0.5, 0.05), 8000 + 10 * E, 0.0)
    st, w, infos, stats = _run(env, "plain", "fp64", pairs, 1, itr)
    assert stats["last_exact_E"] == E
    _check(pairs, w, infos, itr, float("inf"), TOL64)


def test_exact_kernel_on_teams(env):
    """Exact E = 25 on teams of 8 CTAs (N = 100000 -> ceil(N / 4096) = 25)."""
    itr = 30
    pairs = _pairs([100000, 99000], (0.05, 0.002), 9100, 1e-4)
    st, w, infos, stats = _run(env, "log", "fp32", pairs, 8, itr)
    assert all(i.team_size == 8 for i in infos)
    assert stats["last_exact_E"] == 25
    _check(pairs, w, infos, itr, 1e10, TOL32)


def test_generic_kernel_masked_chunks(env):
    """Pairs of E = 2, 13, 27 and 32 in one launch take the generic kernel; 2,
    13 and 27 end in a chunk with identity steps."""
    itr = 40
    pairs = _pairs([_n_for(E) for E in (2, 13, 27, 32)], (0.4, 0.1, 0.02, 0.005), 9200, 1e-3)
    st, w, infos, stats = _run(env, "log", "fp32", pairs, 1, itr)
    assert stats["last_exact_E"] == 0 and stats["exact_launches"] == 0
    _check(pairs, w, infos, itr, 1e10, TOL32)


def test_exact_and_generic_agree(env):
    """The same pairs through the exact kernel (alone) and the generic one (with
    a pair of another point count in the launch)."""
    itr = 60
    pairs = _pairs([_n_for(27, k) for k in range(3)], (0.2, 0.03, 0.004), 9300, 1e-3)
    _, w_x, i_x, s_x = _run(env, "log", "fp32", pairs, 1, itr)
    extra = _pairs([_n_for(9)], (0.1,), 9399, 1e-3)
    _, w_g, i_g, s_g = _run(env, "log", "fp32", pairs + extra, 1, itr)
    assert s_x["last_exact_E"] == 27 and s_g["last_exact_E"] == 0
    for k in range(3):
        assert i_x[k].iters == i_g[k].iters == itr
        assert abs(w_x[k] - w_g[k]) <= 1e-5 * abs(w_g[k]), (k, w_x[k], w_g[k])
    _check(pairs, np.asarray(w_x), i_x, itr, 1e10, TOL32)


def test_graph_key_separates_point_counts(env):
    """Two batches with the same count, team size and header size but pairs of
    10 and of 12 points per thread: the second must not replay the graph
    captured for the first (the exact instantiation is part of the key)."""
    torch, fs1 = env
    itr = 30
    p10 = _pairs([_n_for(10, k) for k in range(3)], (0.2, 0.05, 0.01), 9500, 1e-3)
    p12 = _pairs([_n_for(12, k) for k in range(3)], (0.2, 0.05, 0.01), 9600, 1e-3)

    def probs_of(pairs):
        keep, probs = [], []
        for a, b, h, eps in pairs:
            ta = torch.tensor(a, dtype=torch.float32, device="cuda")
            tb = torch.tensor(b, dtype=torch.float32, device="cuda")
            keep += [ta, tb]
            probs.append(fs1.Solver.problem(ta, tb, h, eps, 0.0, itr))
        return keep, probs

    k10, q10 = probs_of(p10)
    k12, q12 = probs_of(p12)
    s = fs1.Solver("log", "fp32", team_size=1, autotune=False)
    s.solve(q10)
    s.solve(q10)                      # captured
    _, w10, i10 = s.solve(q10)        # replayed
    st = s.stats()
    assert st["graphs_captured"] == 1 and st["graph_replays"] == 2 and st["last_exact_E"] == 10
    _, w12, i12 = s.solve(q12)        # another signature: direct launch of E = 12
    st2 = s.stats()
    s.close()
    assert st2["graph_replays"] == 2 and st2["last_exact_E"] == 12
    assert all(i.status == fs1.FS1_ENOTCONV for i in i12)
    _check(p10, w10, i10, itr, 1e10, TOL32)
    _check(p12, w12, i12, itr, 1e10, TOL32)
