"""3D grids: Algorithm 2 with a third axis (the extension stated by the closing
remark of Section 4), against the FP64 oracle."""
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


def _solve(env, probs, **kw):
    torch, fs1 = env
    s = fs1.Solver("log", "fp32", **kw)
    keep, ps = [], []
    for (a, b, h, eps, tol, itr) in probs:
        ta = torch.tensor(a, dtype=torch.float64, device="cuda")
        tb = torch.tensor(b, dtype=torch.float64, device="cuda")
        keep += [ta, tb]
        ps.append(fs1.Solver.problem(ta, tb, h, eps, tol, itr))
    st, w, infos = s.solve(ps)
    s.close()
    return w, infos


def _rand(seed, shape, floor=0.02):
    rng = np.random.default_rng(seed)
    a = rng.uniform(0, 1, shape) + floor
    b = rng.uniform(0, 1, shape) + floor
    return a / a.sum(), b / b.sum()


def _h(shape):
    ns, nm, nf = shape
    return (1.0 / nf, 1.0 / nm, 1.0 / ns)


# c P = (h / eps) ceil(L / 32) <= 40 takes the FP32-frame line scan on an axis;
# the last two shapes take the extended-range scan on some or all axes.
# (6, 200, 64), 5e-4: the extended-range scan on all three axes, with 64- and
# 200-point lines
@pytest.mark.parametrize("shape,eps", [((4, 5, 6), 0.05), ((3, 17, 33), 0.02), ((7, 9, 40), 0.01),
                                       ((1, 8, 9), 0.05), ((12, 1, 20), 0.05), ((5, 6, 7), 1e-3),
                                       ((6, 40, 8), 2e-3), ((6, 200, 64), 5e-4)])
def test_3d_against_oracle(env, shape, eps):
    _, fs1 = env
    a, b = _rand(sum(shape) * 31 + 7, shape)
    h = _h(shape)
    itr = 40
    w, infos = _solve(env, [(a, b, h, eps, 0.0, itr)])
    ref = cref.solve(a, b, h, eps, 0.0, itr, tau=1e10)
    assert infos[0].status in (fs1.FS1_OK, fs1.FS1_ENOTCONV)
    assert infos[0].iters == ref.iters == itr
    assert abs(w[0] - ref.w) <= TOL32 * abs(ref.w), (shape, eps, w[0], ref.w)
    assert abs(infos[0].marginal_err - ref.err) <= 1e-3 * ref.err + 1e-7


def test_3d_product_equals_three_1d(env):
    """Separable inputs: after the first iteration W_3D = W_x + W_y + W_z."""
    torch, fs1 = env
    a3, b3, ((ax, bx), (ay, by), (az, bz)) = inputs.product_pair_3d(2, 24, 10, 7)
    h, eps, itr = (1 / 24, 1 / 10, 1 / 7), 0.04, 30
    w3, i3 = _solve(env, [(a3, b3, h, eps, 0.0, itr)])
    w1, i1 = _solve(env, [(p, q, hh, eps, 0.0, itr) for (p, q), hh in zip(((ax, bx), (ay, by), (az, bz)), h)])
    assert abs(w3[0] - sum(w1)) <= TOL32 * w3[0]


def test_3d_and_2d_in_one_launch(env):
    probs = []
    for i, shape in enumerate([(5, 8, 9), (12, 16), (3, 4, 40), (20, 7)]):
        a, b = _rand(500 + i, shape)
        h = _h(shape) if len(shape) == 3 else (1.0 / shape[1], 1.0 / shape[0])
        probs.append((a, b, h, 0.03, 1e-5, 2000))
    w, infos = _solve(env, probs)
    _, fs1 = env
    for (a, b, h, eps, tol, itr), info, wi in zip(probs, infos, w):
        assert info.status == fs1.FS1_OK and info.marginal_err <= tol
        ref = cref.solve(a, b, h, eps, 0.0, info.iters, tau=1e10)
        assert abs(wi - ref.w) <= TOL32 * abs(ref.w)
        ro = cref.solve(a, b, h, eps, tol, itr, tau=1e10)
        assert abs(ro.iters - info.iters) <= 1


def test_3d_64cube_sampled(env):
    """A 64^3 grid (262144 points, as many as one 512^2 image) for 15
    iterations, against the oracle."""
    shape = (64, 64, 64)
    a, b = _rand(99, shape)
    h, eps, itr = _h(shape), 0.02, 15
    w, infos = _solve(env, [(a, b, h, eps, 0.0, itr)])
    ref = cref.solve(a, b, h, eps, 0.0, itr, tau=1e10)
    assert infos[0].iters == itr
    assert abs(w[0] - ref.w) <= TOL32 * abs(ref.w)
    assert abs(infos[0].marginal_err - ref.err) <= 1e-3 * ref.err


def test_3d_warm_start_resume_bit_identical(env):
    torch, fs1 = env
    a, b = _rand(77, (6, 10, 12))
    h, eps = _h((6, 10, 12)), 0.02
    ta = torch.tensor(a, device="cuda")
    tb = torch.tensor(b, device="cuda")
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


def test_3d_axis_above_limit_unsupported(env):
    _, fs1 = env
    a, b = _rand(3, (2, 1025, 2))
    w, infos = _solve(env, [(a, b, (0.5, 1 / 1025, 0.5), 0.05, 0.0, 5)])
    assert infos[0].status == fs1.FS1_EUNSUPPORTED
