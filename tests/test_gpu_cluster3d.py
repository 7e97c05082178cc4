"""3D grids resident in one thread-block cluster (the separable extension of
the closing remark of Section 4, K = K_slow (x) K_mid (x) K_fast; Algorithm 2
with a third axis), against the FP64 oracle and against the grid kernel on the
same inputs.

Tolerances as the other grid tests: relative W <= 1e-4 and marginal error
<= 1e-3 relative at equal iteration counts (FP32 stabilised against FP64)."""
import numpy as np
import pytest

from oracle import cref

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


def _rand(seed, shape, floor=0.02):
    rng = np.random.default_rng(seed)
    a = rng.uniform(0, 1, shape) + floor
    b = rng.uniform(0, 1, shape) + floor
    return a / a.sum(), b / b.sum()


def _h(shape):
    ns, nm, nf = shape
    return (1.0 / nf, 1.0 / nm, 1.0 / ns)


def _solve(env, probs, grid=False, pots=False):
    """Solve probs = [(a, b, h, eps, tol, itr)] in one call; pots: also return
    the log potentials f, g of each problem (host arrays)."""
    torch, fs1 = env
    s = fs1.Solver("log", "fp32", grid2d=grid)
    keep, ps, fg = [], [], []
    for (a, b, h, eps, tol, itr) in probs:
        ta = torch.tensor(a, dtype=torch.float64, device="cuda")
        tb = torch.tensor(b, dtype=torch.float64, device="cuda")
        keep += [ta, tb]
        f = g = None
        if pots:
            f = torch.empty_like(ta)
            g = torch.empty_like(ta)
            fg.append((f, g))
        ps.append(fs1.Solver.problem(ta, tb, h, eps, tol, itr, f_out=f, g_out=g))
    st, w, infos = s.solve(ps)
    s.close()
    return w, infos, [(f.cpu().numpy(), g.cpu().numpy()) for f, g in fg]


# every axis with h / eps <= 8; the shapes cover a middle axis that is not a
# multiple of 8, odd fast axes, one plane, slow axes that leave the last CTAs
# of the cluster empty or hold up to 7 planes per CTA, and the 64^3 grid of
# the 3D benchmark at c = 7.8
SHAPES = [((4, 5, 6), 0.05), ((16, 16, 16), 0.01), ((33, 24, 50), 6e-3), ((1, 8, 9), 0.05),
          ((10, 20, 63), 0.013), ((100, 9, 3), 0.045), ((64, 64, 64), 2e-3)]


@pytest.mark.parametrize("shape,eps", SHAPES)
def test_cluster3d_against_oracle(env, shape, eps):
    _, fs1 = env
    a, b = _rand(sum(shape) * 17 + 3, shape)
    h = _h(shape)
    itr = 15 if np.prod(shape) > 100000 else 40
    w, infos, _ = _solve(env, [(a, b, h, eps, 0.0, itr)])
    ref = cref.solve(a, b, h, eps, 0.0, itr, tau=1e10)
    assert infos[0].team_size >= 8, "the cluster kernel took the grid"
    assert infos[0].status in (fs1.FS1_OK, fs1.FS1_ENOTCONV)
    assert infos[0].iters == ref.iters == itr
    assert abs(w[0] - ref.w) <= TOL32 * abs(ref.w), (shape, w[0], ref.w)
    assert abs(infos[0].marginal_err - ref.err) <= 1e-3 * ref.err + 1e-7


@pytest.mark.parametrize("shape,eps", [((33, 24, 50), 6e-3), ((10, 20, 63), 0.013), ((64, 64, 64), 2e-3)])
def test_cluster3d_matches_grid_kernel(env, shape, eps):
    """The cluster kernel and the grid kernel run the same iteration: W, the
    marginal error and the returned potentials agree point by point."""
    a, b = _rand(sum(shape) + 11, shape)
    p = [(a, b, _h(shape), eps, 0.0, 30)]
    wc, ic, pc = _solve(env, p, pots=True)
    wg, ig, pg = _solve(env, p, grid=True, pots=True)
    assert ic[0].team_size >= 8 and ig[0].team_size == 0
    assert ic[0].iters == ig[0].iters == 30
    assert abs(wc[0] - wg[0]) <= TOL32 * abs(wg[0])
    assert abs(ic[0].marginal_err - ig[0].marginal_err) <= 1e-3 * ig[0].marginal_err
    (fc, gc), (fg, gg) = pc[0], pg[0]
    assert np.max(np.abs(fc - fg)) <= 1e-3 and np.max(np.abs(gc - gg)) <= 1e-3


def test_cluster3d_stop_rule(env):
    """Algorithm 2's while condition: each grid stops within one iteration of
    the oracle's own stop, with W matching the oracle at the GPU's count."""
    _, fs1 = env
    probs = []
    for i, (shape, eps) in enumerate([((4, 5, 6), 0.05), ((16, 16, 16), 0.02), ((9, 24, 40), 0.02)]):
        a, b = _rand(700 + i, shape)
        probs.append((a, b, _h(shape), eps, 1e-5, 3000))
    w, infos, _ = _solve(env, probs)
    for (a, b, h, eps, tol, itr), info, wi in zip(probs, infos, w):
        assert info.team_size >= 8
        assert info.status == fs1.FS1_OK and info.marginal_err <= tol
        ro = cref.solve(a, b, h, eps, tol, itr, tau=1e10)
        assert abs(ro.iters - info.iters) <= 1
        ref = cref.solve(a, b, h, eps, 0.0, info.iters, tau=1e10)
        assert abs(wi - ref.w) <= TOL32 * abs(ref.w)


def test_cluster3d_warm_start_resume_bit_identical(env):
    """20 iterations, then 30 more from the returned potentials, equal 50 in
    one call exactly (W and the marginal error)."""
    torch, fs1 = env
    shape = (6, 10, 12)
    a, b = _rand(77, shape)
    h, eps = _h(shape), 0.03
    ta = torch.tensor(a, device="cuda")
    tb = torch.tensor(b, device="cuda")
    s = fs1.Solver("log", "fp32")
    st, w_full, i_full = s.solve([fs1.Solver.problem(ta, tb, h, eps, 0.0, 50)])
    f = torch.empty_like(ta)
    g = torch.empty_like(ta)
    s.solve([fs1.Solver.problem(ta, tb, h, eps, 0.0, 20, f_out=f, g_out=g)])
    st, w_res, i_res = s.solve([fs1.Solver.problem(ta, tb, h, eps, 0.0, 30, f_init=f, g_init=g)])
    s.close()
    assert i_full[0].team_size >= 8 and i_res[0].team_size >= 8
    assert i_res[0].iters == 30
    assert w_res[0] == w_full[0]
    assert i_res[0].marginal_err == i_full[0].marginal_err


def test_cluster3d_no_iterations(env):
    """itr_max = 0: the initial iterate u = v = 1 / N, its cost and error."""
    shape = (8, 12, 20)
    a, b = _rand(5, shape)
    w, infos, _ = _solve(env, [(a, b, _h(shape), 0.02, 0.0, 0)])
    ref = cref.solve(a, b, _h(shape), 0.02, 0.0, 0, tau=1e10)
    assert infos[0].iters == 0 and infos[0].team_size >= 8
    assert abs(w[0] - ref.w) <= TOL32 * abs(ref.w)
    assert abs(infos[0].marginal_err - ref.err) <= 1e-3 * ref.err


def test_cluster3d_many_grids_one_call(env):
    """More grids than clusters fit at once, of several cluster sizes, from
    one queue per size; each against the oracle."""
    rng = np.random.default_rng(42)
    probs = []
    for i in range(24):
        shape = (int(rng.integers(1, 40)), int(rng.integers(2, 33)), int(rng.integers(1, 65)))
        eps = 1.0 / (7.5 * min(shape[1], shape[2] if shape[2] > 1 else 99, shape[0] if shape[0] > 1 else 99))
        a, b = _rand(900 + i, shape)
        probs.append((a, b, _h(shape), eps, 0.0, 25))
    w, infos, _ = _solve(env, probs)
    refs = cref.solve_many(probs, tau=1e10)
    for k, (info, wi, r) in enumerate(zip(infos, w, refs)):
        assert info.team_size >= 8, k
        assert info.iters == r.iters == 25
        assert abs(wi - r.w) <= TOL32 * abs(r.w), (k, probs[k][0].shape, wi, r.w)
        assert abs(info.marginal_err - r.err) <= 1e-3 * r.err + 1e-7


def test_cluster3d_blob_inputs_long_run(env):
    """The 3D benchmark's inputs (Gaussian blobs over a 1e-7 floor: masses over
    seven decades; c = 7.8 on every axis) make the scalings span hundreds of
    binary orders within a few points: 20 iterations against the oracle, and
    300 against the grid kernel (W, marginal error, potentials point by
    point)."""
    from paper_2202_10042_gb300 import inputs
    p = inputs.workload9(0)
    h = tuple(p.h)
    w, infos, _ = _solve(env, [(p.a, p.b, h, p.eps, 0.0, 20)])
    ref = cref.solve(p.a, p.b, h, p.eps, 0.0, 20, tau=1e10)
    assert infos[0].team_size >= 8
    assert abs(w[0] - ref.w) <= TOL32 * abs(ref.w)
    assert abs(infos[0].marginal_err - ref.err) <= 1e-3 * ref.err
    q = [(p.a, p.b, h, p.eps, 0.0, 300)]
    wc, ic, pc = _solve(env, q, pots=True)
    wg, ig, pg = _solve(env, q, grid=True, pots=True)
    assert ic[0].team_size >= 8 and ig[0].team_size == 0
    assert abs(wc[0] - wg[0]) <= TOL32 * abs(wg[0])
    assert abs(ic[0].marginal_err - ig[0].marginal_err) <= 1e-3 * ig[0].marginal_err
    (fc, gc), (fg, gg) = pc[0], pg[0]
    assert np.max(np.abs(fc - fg)) <= 1e-3 and np.max(np.abs(gc - gg)) <= 1e-3
