"""Stabilised 1D pairs beyond the team kernel's on-chip capacity: the solve
with the state in device memory (chunks of 8192 points, one launch per
half-step shared by up to 8 pairs) against the FP64 oracle at the GPU's
iteration count.  Tolerance: relative W1 1e-4 (FP32 variant)."""
import numpy as np
import pytest

from oracle import cref
from paper_2202_10042_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL32 = 1e-4
# one more 512-thread CTA of 32 points than a GB300's 152 SMs hold
N_BEYOND = 152 * 512 * 32 + 512 * 32 + 1234


@pytest.fixture(scope="module")
def env():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2202_10042_gb300 import fs1
    fs1.load()
    return torch, fs1


def _pair(index, n, c, floor=1e-3):
    """FP32-rounded pair on [0, 1] with eps = h / c (h = 1 / n)."""
    a, b = inputs.random_pair_1d(index, n, floor=floor)
    a = a.astype(np.float32).astype(np.float64)
    b = b.astype(np.float32).astype(np.float64)
    return a, b, 1.0 / n, 1.0 / (c * n)


def _solve(env, pairs, itr, tol=0.0, outs=None, inits=None):
    torch, fs1 = env
    keep, probs = [], []
    for k, (a, b, h, eps) in enumerate(pairs):
        ta = torch.tensor(a, dtype=torch.float32, device="cuda")
        tb = torch.tensor(b, dtype=torch.float32, device="cuda")
        keep += [ta, tb]
        kw = {}
        if outs is not None:
            kw.update(f_out=outs[k][0], g_out=outs[k][1])
        if inits is not None:
            kw.update(f_init=inits[k][0], g_init=inits[k][1])
        probs.append(fs1.Solver.problem(ta, tb, h, eps, tol, itr, **kw))
    s = fs1.Solver("log", "fp32", autotune=False)
    st, w, infos = s.solve(probs)
    s.close()
    return st, w, infos


def _ref(pair, itr, tol=0.0):
    a, b, h, eps = pair
    return cref.solve(a, b, h, eps, tol, itr, tau=1e10)


def test_stream_beyond_capacity_against_oracle(env):
    torch, fs1 = env
    pair = _pair(31, N_BEYOND, 0.02)
    st, w, infos = _solve(env, [pair], 20)
    assert infos[0].status == fs1.FS1_ENOTCONV and infos[0].iters == 20 and infos[0].team_size == 0
    ref = _ref(pair, 20)
    assert abs(w[0] - ref.w) <= TOL32 * abs(ref.w), (w[0], ref.w)
    assert abs(infos[0].marginal_err - ref.err) <= 1e-3 * ref.err + 1e-6


def test_stream_forced_by_the_frame_rule(env):
    """h / eps = 4.8 allows 5 points per thread: a million points exceed the
    152 co-resident CTAs and take the streaming path."""
    torch, fs1 = env
    pair = _pair(32, 1_000_003, 4.8)
    st, w, infos = _solve(env, [pair], 15)
    assert infos[0].team_size == 0 and infos[0].iters == 15
    ref = _ref(pair, 15)
    assert abs(w[0] - ref.w) <= TOL32 * abs(ref.w), (w[0], ref.w)


def test_stream_stop_rule(env):
    torch, fs1 = env
    pair = _pair(33, N_BEYOND, 1e-4)   # the oracle stops at iteration 21
    st, w, infos = _solve(env, [pair], 300, tol=1e-3)
    i = infos[0]
    assert i.status == fs1.FS1_OK and i.marginal_err <= 1e-3 and i.iters < 300
    stop = _ref(pair, 300, tol=1e-3)
    assert abs(i.iters - stop.iters) <= 1
    ref = _ref(pair, int(i.iters))
    assert abs(w[0] - ref.w) <= TOL32 * abs(ref.w)


def test_stream_pair_in_a_mixed_batch(env):
    """A pair beyond the capacity and two small ones in one call: the small ones
    run on the team kernel, the large one streams; all match the oracle."""
    torch, fs1 = env
    pairs = [_pair(34, 5000, 0.1), _pair(35, N_BEYOND, 0.05), _pair(36, 70000, 0.01)]
    st, w, infos = _solve(env, pairs, 12)
    assert infos[1].team_size == 0 and infos[0].team_size >= 1 and infos[2].team_size >= 1
    refs = cref.solve_many([(a, b, h, eps, 0.0, 12) for a, b, h, eps in pairs], tau=1e10)
    for k, r in enumerate(refs):
        assert infos[k].iters == 12
        assert abs(w[k] - r.w) <= TOL32 * abs(r.w), (k, w[k], r.w)


def test_stream_warm_start_resume_bit_identical(env):
    torch, fs1 = env
    pair = _pair(37, N_BEYOND, 0.03)
    n = pair[0].size
    st, w_full, i_full = _solve(env, [pair], 20)
    f = torch.empty(n, dtype=torch.float64, device="cuda")
    g = torch.empty_like(f)
    _solve(env, [pair], 12, outs=[(f, g)])
    assert bool(torch.isfinite(f).all()) and bool(torch.isfinite(g).all())
    st, w_res, i_res = _solve(env, [pair], 8, inits=[(f, g)])
    assert i_res[0].iters == 8
    assert w_res[0] == w_full[0]
    assert i_res[0].marginal_err == i_full[0].marginal_err


def test_stream_input_check(env):
    """A negative mass or unequal totals in a pair that would stream is refused
    with FS1_EINVAL by the chunked device check; a valid pair in the same call
    is solved."""
    torch, fs1 = env
    a, b, h, eps = _pair(38, N_BEYOND, 0.05)
    a_neg = a.copy()
    a_neg[N_BEYOND - 7] = -1e-9
    b_big = b * 1.01
    small = _pair(39, 3000, 0.1)
    st, w, infos = _solve(env, [(a_neg, b, h, eps), (a, b_big, h, eps), small], 5)
    assert infos[0].status == fs1.FS1_EINVAL and infos[1].status == fs1.FS1_EINVAL
    assert infos[2].status == fs1.FS1_ENOTCONV
    ref = cref.solve(*small[:2], small[2], small[3], 0.0, 5, tau=1e10)
    assert abs(w[2] - ref.w) <= TOL32 * abs(ref.w)


def test_stream_pairs_share_launches(env):
    """Ten streamed pairs in one call (two groups of shared launches: 8 and 2)
    ending at different iterations (caps, and one meeting tol), and one
    refused by the input check: every pair gives the same bits as alone, and
    two match the oracle."""
    torch, fs1 = env
    # h / eps = 4.8 allows 5 points per thread: 390 000 points and more stream
    pairs = [_pair(60 + k, 400_000 + 7919 * k, 4.8) for k in range(9)] + [_pair(33, N_BEYOND, 1e-4)]
    caps = [120, 40, 77, 100, 13, 120, 64, 90, 31, 300]
    tols = [0.0] * 9 + [1e-3]   # the last pair stops at iteration 21 (as alone)
    bad_a = pairs[3][0].copy()
    bad_a[100] = -1e-6
    pairs.insert(4, (bad_a, pairs[3][1], pairs[3][2], pairs[3][3]))
    caps.insert(4, 50)
    tols.insert(4, 0.0)
    keep, probs = [], []
    for (a, b, h, eps), cap, tol in zip(pairs, caps, tols):
        ta = torch.tensor(a, dtype=torch.float32, device="cuda")
        tb = torch.tensor(b, dtype=torch.float32, device="cuda")
        keep += [ta, tb]
        probs.append(fs1.Solver.problem(ta, tb, h, eps, tol, cap))
    s = fs1.Solver("log", "fp32", autotune=False)
    _, w, infos = s.solve(probs)
    s.close()
    assert infos[4].status == fs1.FS1_EINVAL
    for k, (pair, cap, tol) in enumerate(zip(pairs, caps, tols)):
        if k == 4:
            continue
        assert infos[k].team_size == 0, k
        _, w1, i1 = _solve(env, [pair], cap, tol=tol)
        assert (w1[0], i1[0].iters, i1[0].marginal_err) == (w[k], infos[k].iters, infos[k].marginal_err), k
        if tol == 0.0:
            assert infos[k].iters == cap and infos[k].status == fs1.FS1_ENOTCONV
    assert infos[-1].status == fs1.FS1_OK and infos[-1].iters < 300
    for k in (1, 5):
        ref = _ref(pairs[k], int(infos[k].iters))
        assert abs(w[k] - ref.w) <= TOL32 * abs(ref.w), (k, w[k], ref.w)


def test_stream_refuses_large_h_over_eps(env):
    """h / eps = 12 allows 2 points per thread on chip, and a streamed run of 16
    points would span e^192, beyond one FP32 frame: a pair of 160 000 points is
    refused (FS1_EUNSUPPORTED) while the call's other pair is solved."""
    torch, fs1 = env
    pairs = [_pair(80, 160_000, 12.0), _pair(81, 3000, 0.1)]
    st, w, infos = _solve(env, pairs, 10)
    assert infos[0].status == fs1.FS1_EUNSUPPORTED
    assert infos[1].status == fs1.FS1_ENOTCONV and infos[1].iters == 10
