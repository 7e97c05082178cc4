"""GPU parity of the 2D FS-1 path (Algorithm 2) against the CPU FP64 oracle.

Tolerance: relative W1 <= 1e-4 (FP32 stabilised), at the GPU's iteration count."""
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


def _solve(env, probs):
    torch, fs1 = env
    s = fs1.Solver("log", "fp32")
    keep, ps = [], []
    for (a2, b2, h, eps, tol, itr) in probs:
        ta = torch.tensor(a2, dtype=torch.float64, device="cuda")
        tb = torch.tensor(b2, dtype=torch.float64, device="cuda")
        keep += [ta, tb]
        ps.append(fs1.Solver.problem(ta, tb, h, eps, tol, itr))
    st, w, infos = s.solve(ps)
    s.close()
    return w, infos


def _rand2d(seed, ns, nf, floor=0.02):
    rng = np.random.default_rng(seed)
    a = rng.uniform(0, 1, (ns, nf)) + floor
    b = rng.uniform(0, 1, (ns, nf)) + floor
    return a / a.sum(), b / b.sum()


# c = h / eps and the points per lane P decide the line scan of an axis:
# c P <= 40 one FP32 frame per lane, else the per-point extended-range scan.
# The first six cases take the frame scan on both axes, the others the
# extended-range scan on both axes or on one of them, over a range of c
# (from about 3 to 300) and line lengths up to 1024.
@pytest.mark.parametrize("ns,nf,eps", [(7, 9, 0.1), (33, 40, 0.02), (64, 64, 0.01), (70, 100, 5e-3),
                                       (1, 50, 0.02), (45, 1, 0.02), (40, 64, 2e-4), (8, 512, 2e-3),
                                       (48, 48, 6.9e-4), (200, 600, 5e-4), (16, 1024, 2e-4)])
def test_2d_against_oracle(env, ns, nf, eps):
    a2, b2 = _rand2d(ns * 1000 + nf, ns, nf)
    h = (1.0 / nf, 1.0 / ns)
    itr = 60
    w, infos = _solve(env, [(a2, b2, h, eps, 0.0, itr)])
    ref = cref.solve(a2, b2, h, eps, 0.0, itr, tau=1e10)
    _, fs1 = env
    assert infos[0].status in (fs1.FS1_OK, fs1.FS1_ENOTCONV)
    assert infos[0].iters == ref.iters == itr
    assert abs(w[0] - ref.w) <= TOL32 * abs(ref.w)
    assert abs(infos[0].marginal_err - ref.err) <= 1e-3 * ref.err + 1e-7


def test_2d_batch_mixed_sizes_and_stop(env):
    probs = []
    for i, (ns, nf) in enumerate([(16, 24), (50, 31), (8, 8), (33, 65)]):
        a2, b2 = _rand2d(100 + i, ns, nf)
        probs.append((a2, b2, (1.0 / nf, 1.0 / ns), 0.05, 1e-5, 3000))
    w, infos = _solve(env, probs)
    _, fs1 = env
    for (a2, b2, h, eps, tol, itr), info, wi in zip(probs, infos, w):
        assert info.status == fs1.FS1_OK and info.marginal_err <= tol
        ref = cref.solve(a2, b2, h, eps, 0.0, info.iters, tau=1e10)
        assert abs(wi - ref.w) <= TOL32 * abs(ref.w)
        ro = cref.solve(a2, b2, h, eps, tol, itr, tau=1e10)
        assert abs(ro.iters - info.iters) <= 1


def test_2d_product_equals_two_1d(env):
    """Section 4: for separable inputs the 2D iterates factor into the 1D ones,
    so after the first iteration W_2D = W_x + W_y (GPU against GPU and oracle)."""
    torch, fs1 = env
    a2, b2, (ax, bx), (ay, by) = inputs.product_pair_2d(3, 48, 40)
    hf, hs, eps, itr = 1 / 48, 1 / 40, 0.03, 40
    w2, i2 = _solve(env, [(a2, b2, (hf, hs), eps, 0.0, itr)])
    s = fs1.Solver("log", "fp32")
    keep, ps = [], []
    for (a, b, h) in ((ax, bx, hf), (ay, by, hs)):
        ta = torch.tensor(a, device="cuda")
        tb = torch.tensor(b, device="cuda")
        keep += [ta, tb]
        ps.append(fs1.Solver.problem(ta, tb, h, eps, 0.0, itr))
    st, w1, i1 = s.solve(ps)
    s.close()
    assert abs(w2[0] - (w1[0] + w1[1])) <= TOL32 * w2[0]


def test_workload4_full_size_sampled(env):
    """Workload 4 at its full size (512 x 512 blobs, eps = 1e-3) with the
    iteration cap cut to 40 so that the FP64 oracle finishes in seconds."""
    ps = [inputs.workload4(i, itr_max=40) for i in (0, 1)]
    probs = [(p.a, p.b, p.h, p.eps, p.tol, p.itr_max) for p in ps]
    w, infos = _solve(env, probs)
    refs = cref.solve_many(probs, tau=1e10)
    for i, r in enumerate(refs):
        assert infos[i].iters == r.iters == 40
        assert abs(w[i] - r.w) <= TOL32 * abs(r.w)
        assert abs(infos[i].marginal_err - r.err) <= 1e-3 * r.err


def test_2d_warm_start_resume_bit_identical(env):
    torch, fs1 = env
    a2, b2 = _rand2d(77, 40, 56)
    h, eps = (1 / 56, 1 / 40), 0.01
    ta = torch.tensor(a2, device="cuda")
    tb = torch.tensor(b2, device="cuda")
    s = fs1.Solver("log", "fp32")
    st, w_full, i_full = s.solve([fs1.Solver.problem(ta, tb, h, eps, 0.0, 50)])
    f = torch.empty_like(ta)
    g = torch.empty_like(ta)
    s.solve([fs1.Solver.problem(ta, tb, h, eps, 0.0, 20, f_out=f, g_out=g)])
    st, w_res, i_res = s.solve([fs1.Solver.problem(ta, tb, h, eps, 0.0, 30, f_init=f, g_init=g)])
    s.close()
    assert i_res[0].iters == 30
    assert w_res[0] == w_full[0]
    assert i_res[0].marginal_err == i_full[0].marginal_err


@pytest.mark.parametrize("ns,nf", [(300, 1024), (1024, 200)])
def test_2d_longest_lines_against_oracle(env, ns, nf):
    """Rows or columns of 1024 points, the longest a line may be."""
    a2, b2 = _rand2d(ns + 7 * nf, ns, nf)
    h, eps, itr = (1.0 / nf, 1.0 / ns), 2e-3, 12
    w, infos = _solve(env, [(a2, b2, h, eps, 0.0, itr)])
    ref = cref.solve(a2, b2, h, eps, 0.0, itr, tau=1e10)
    assert infos[0].iters == ref.iters == itr
    assert abs(w[0] - ref.w) <= TOL32 * abs(ref.w)
    assert abs(infos[0].marginal_err - ref.err) <= 1e-3 * ref.err


def test_2d_side_above_limit_unsupported(env):
    _, fs1 = env
    a2, b2 = _rand2d(3, 1025, 4)
    w, infos = _solve(env, [(a2, b2, (0.25, 1 / 1025), 0.05, 0.0, 5)])
    assert infos[0].status == fs1.FS1_EUNSUPPORTED


def test_workload4_full_length_against_stored_oracle(env):
    """Workload 4 to its own stop (tol 1e-6, cap 5000) in one launch, against
    the FP64 oracle's values stored by tests/golden/make_workload4_oracle.py:
    two images that reach the cap and one that stops early (Algorithm 2's
    while condition; the stop within one iteration)."""
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "workload4_oracle.json")) as fh:
        gold = json.load(fh)["images"]
    idx = sorted(int(k) for k in gold)
    ps = [inputs.workload4(i) for i in idx]
    w, infos = _solve(env, [(p.a, p.b, tuple(p.h), p.eps, p.tol, p.itr_max) for p in ps])
    _, fs1 = env
    for k, i in enumerate(idx):
        g = gold[str(i)]
        if g["iters"] == g["itr_max"]:
            assert infos[k].iters == g["iters"] and infos[k].status == fs1.FS1_ENOTCONV
            assert abs(infos[k].marginal_err - g["err"]) <= 1e-3 * g["err"] + 1e-7
        else:
            assert infos[k].status == fs1.FS1_OK and abs(infos[k].iters - g["iters"]) <= 1
            assert infos[k].marginal_err <= g["tol"]
        assert abs(w[k] - g["w"]) <= TOL32 * abs(g["w"]), (i, w[k], g["w"])
