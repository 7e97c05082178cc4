"""FS1_VARIANT_PAPER: the stabilised FS-1 of the Remarks in Sections 2 and 3 as
written (FP64, tau-triggered absorption into A = alpha/eps, B = beta/eps,
per-point factors lam e^{+-(S_{k+1}-S_k)}), against the FP64 oracle's same form."""
import math

import numpy as np
import pytest

from oracle import cref
from paper_2202_10042_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL64 = 1e-6


@pytest.fixture(scope="module")
def env():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2202_10042_gb300 import fs1
    fs1.load()
    return torch, fs1


def _solve(env, pairs, tau=1e10, variant="paper", prec="fp64", outs=False):
    torch, fs1 = env
    s = fs1.Solver(variant, prec, tau=tau)
    keep, probs, fg = [], [], []
    for (a, b, h, eps, tol, itr) in pairs:
        ta = torch.tensor(a, dtype=torch.float64, device="cuda")
        tb = torch.tensor(b, dtype=torch.float64, device="cuda")
        f = torch.empty_like(ta) if outs else None
        g = torch.empty_like(ta) if outs else None
        keep += [ta, tb]
        fg.append((f, g))
        probs.append(fs1.Solver.problem(ta, tb, h, eps, tol, itr, f_out=f, g_out=g))
    st, w, infos = s.solve(probs)
    s.close()
    return w, infos, fg


def _pair(n, index, floor=1e-3):
    return inputs.random_pair_1d(index, n, floor=floor)


@pytest.mark.parametrize("tau", [1e3, 1e10])
@pytest.mark.parametrize("n,eps,itr", [(37, 0.05, 200), (500, 0.01, 300), (2000, 1e-3, 200), (9000, 2e-3, 100)])
def test_paper_form_against_oracle(env, tau, n, eps, itr):
    _, fs1 = env
    a, b = _pair(n, n + int(1 / eps))
    w, infos, _ = _solve(env, [(a, b, 1.0 / n, eps, 0.0, itr)], tau=tau)
    ref = cref.solve(a, b, 1.0 / n, eps, 0.0, itr, tau=tau)
    assert infos[0].status == fs1.FS1_ENOTCONV and infos[0].iters == ref.iters == itr
    assert abs(w[0] - ref.w) <= TOL64 * abs(ref.w), (w[0], ref.w)
    assert abs(infos[0].marginal_err - ref.err) <= 1e-6 * ref.err + 1e-14


def test_paper_form_stop_rule(env):
    _, fs1 = env
    a, b = _pair(800, 3)
    w, infos, _ = _solve(env, [(a, b, 1 / 800, 0.02, 1e-9, 5000)], tau=1e6)
    ref = cref.solve(a, b, 1 / 800, 0.02, 1e-9, 5000, tau=1e6)
    assert infos[0].status == fs1.FS1_OK and infos[0].marginal_err <= 1e-9
    assert abs(infos[0].iters - ref.iters) <= 1
    assert abs(w[0] - ref.w) <= TOL64 * abs(ref.w)


def test_paper_form_survives_where_plain_overflows(env):
    """Section 5.2: the Ricker pair at N = 2000, eps = 5e-4 overflows the plain
    FP64 iteration; the absorbed form runs all iterations and matches the
    oracle's absorbed form."""
    _, fs1 = env
    p = inputs.paper_e2(0, n=2000, eps=5e-4)
    pr = [(p.a, p.b, p.h[0], p.eps, 0.0, 500)]
    w, infos, _ = _solve(env, pr, variant="plain", prec="fp64")
    assert infos[0].status == fs1.FS1_ENUMERIC
    w, infos, _ = _solve(env, pr, tau=1e10)
    ref = cref.solve(p.a, p.b, p.h[0], p.eps, 0.0, 500, tau=1e10)
    assert infos[0].status == fs1.FS1_ENOTCONV and infos[0].iters == 500
    assert abs(w[0] - ref.w) <= TOL64 * abs(ref.w), (w[0], ref.w)


def test_paper_form_batch_and_potentials(env):
    pairs = []
    for i, (n, eps) in enumerate([(100, 0.05), (1234, 0.005), (4096, 0.002), (16384, 0.01)]):
        a, b = _pair(n, 50 + i)
        pairs.append((a, b, 1.0 / n, eps, 0.0, 60))
    w, infos, fg = _solve(env, pairs, tau=1e4, outs=True)
    for (a, b, h, eps, tol, itr), wi, info, (f, g) in zip(pairs, w, infos, fg):
        ref = cref.solve(a, b, h, eps, 0.0, itr, tau=1e4, potentials=True)
        assert info.iters == itr and abs(wi - ref.w) <= TOL64 * abs(ref.w)
        fd, gd = f.cpu().numpy(), g.cpu().numpy()
        assert np.max(np.abs(fd - ref.f) / (1 + np.abs(ref.f))) < 1e-9
        assert np.max(np.abs(gd - ref.g) / (1 + np.abs(ref.g))) < 1e-9


def test_paper_form_rejects(env):
    torch, fs1 = env
    a, b = _pair(64, 1)
    a0 = a.copy()
    a0[5] = 0.0
    a0 /= a0.sum()
    big_a, big_b = _pair(16385, 2)
    w, infos, _ = _solve(env, [(a0, b, 1 / 64, 0.05, 0.0, 10), (big_a, big_b, 1 / 16385, 0.05, 0.0, 10),
                               (a, b, 1 / 64, 0.05, 0.0, 10)])
    assert infos[0].status == fs1.FS1_EINVAL          # the stabilised form needs a, b > 0
    assert infos[1].status == fs1.FS1_EUNSUPPORTED    # more points than one CTA holds
    assert infos[2].status == fs1.FS1_ENOTCONV
    a2 = np.full((4, 4), 1 / 16)
    ta = torch.tensor(a2, device="cuda")
    s = fs1.Solver("paper", "fp64")
    st, w, infos = s.solve([fs1.Solver.problem(ta, ta, (0.25, 0.25), 0.1, 0.0, 5)])
    s.close()
    assert infos[0].status == fs1.FS1_EUNSUPPORTED
    with pytest.raises(RuntimeError):
        fs1.Solver("paper", "fp32")
