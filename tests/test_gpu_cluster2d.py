"""The cluster-resident 2D solver (an image in the shared memory of one
16-CTA thread-block cluster) against the CPU FP64 oracle, and against the
grid kernel that keeps the state in device memory (fs1_config.grid2d = 1).

Tolerances: relative W1 <= 1e-4 and marginal error within 1e-3 relative of
the oracle (FP32 stabilised), at the GPU's iteration count."""
import numpy as np
import pytest

from oracle import cref, marginals
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


def _rand2d(seed, ns, nf, floor=0.02):
    rng = np.random.default_rng(seed)
    a = rng.uniform(0, 1, (ns, nf)) + floor
    b = rng.uniform(0, 1, (ns, nf)) + floor
    return a / a.sum(), b / b.sum()


def _solve(env, probs, grid2d=False, outs=False, inits=None):
    torch, fs1 = env
    s = fs1.Solver("log", "fp32", grid2d=grid2d)
    keep, ps, pots = [], [], []
    for k, (a2, b2, h, eps, tol, itr) in enumerate(probs):
        ta = torch.tensor(a2, dtype=torch.float64, device="cuda")
        tb = torch.tensor(b2, dtype=torch.float64, device="cuda")
        keep += [ta, tb]
        kw = {}
        if outs:
            f, g = torch.empty_like(ta), torch.empty_like(ta)
            pots.append((f, g))
            kw.update(f_out=f, g_out=g)
        if inits is not None:
            kw.update(f_init=inits[k][0], g_init=inits[k][1])
        ps.append(fs1.Solver.problem(ta, tb, h, eps, tol, itr, **kw))
    st, w, infos = s.solve(ps)
    s.close()
    return w, infos, pots


def _check_oracle(w, info, a2, b2, h, eps, itr):
    ref = cref.solve(a2, b2, h, eps, 0.0, itr, tau=1e10)
    assert info.iters == ref.iters   # itr, or 0 when the initial error is exactly 0 (one point)
    assert abs(w - ref.w) <= TOL32 * abs(ref.w), (w, ref.w)
    assert abs(info.marginal_err - ref.err) <= 1e-3 * ref.err + 1e-7, (info.marginal_err, ref.err)


def _cluster_holds(ns, nf, h, eps):
    """The cluster kernel takes images of at most 512 x 512 points whose axes
    of more than one point have c = h / eps <= 8; the grid kernel the rest."""
    return (nf == 1 or h[0] / eps <= 8.0) and (ns == 1 or h[1] / eps <= 8.0) and ns <= 512 and nf <= 512


# shapes over the three instantiations (rows of <= 128, 256, 512 points;
# <= 8, 16, 32 rows per CTA), ragged row counts (the last CTAs of the
# cluster partly or wholly empty), single rows and columns, c = h / eps up to
# the frame limit 8, and images beyond it that the grid kernel takes
@pytest.mark.parametrize("ns,nf,eps", [
    (1, 1, 0.05), (1, 37, 0.02), (29, 1, 0.02), (5, 3, 0.1),
    (16, 128, 0.01), (17, 129, 0.01), (100, 256, 2e-3), (160, 160, 1e-2),
    (257, 300, 2e-3), (512, 512, 1e-3), (300, 512, 1e-3), (512, 40, 4e-3),
    (64, 64, 2e-3),            # c = 7.8 on both axes: the largest the frames take
    (64, 64, 1e-3),            # c = 15.6: the grid kernel
    (40, 200, 2e-3),           # c_fast = 2.5, c_slow = 12.5: the grid kernel
])
def test_cluster_against_oracle(env, ns, nf, eps):
    a2, b2 = _rand2d(ns * 7919 + nf, ns, nf)
    h = (1.0 / nf, 1.0 / ns)
    itr = 30
    w, infos, _ = _solve(env, [(a2, b2, h, eps, 0.0, itr)])
    _, fs1 = env
    assert (infos[0].team_size > 0) == _cluster_holds(ns, nf, h, eps)   # CTAs of the cluster, 0: grid kernel
    assert infos[0].status in (fs1.FS1_OK, fs1.FS1_ENOTCONV)
    _check_oracle(w[0], infos[0], a2, b2, h, eps, itr)


def test_cluster_potentials_and_marginals(env):
    """Potentials out, entry by entry, on a ragged shape (both frame paths)."""
    ns, nf, eps, itr = 150, 230, 4e-3, 25
    a2, b2 = _rand2d(5, ns, nf)
    h = (1.0 / nf, 1.0 / ns)
    w, infos, pots = _solve(env, [(a2, b2, h, eps, 0.0, itr)], outs=True)
    assert infos[0].team_size > 0
    f, g = (t.cpu().numpy() for t in pots[0])
    ref = cref.solve(a2, b2, h, eps, 0.0, itr, tau=1e10, potentials=True)
    k = float(np.median(f - ref.f))
    assert abs(k) < 1e-2
    assert np.max(np.abs(f - k - ref.f)) < 1e-3
    assert np.max(np.abs(g + k - ref.g)) < 1e-3
    cs = [h[0] / eps, h[1] / eps]
    row = marginals.row_marginal(f, g, cs)
    assert np.max(np.abs(row - a2) / a2) < 1e-4
    assert abs(marginals.marginal_error(f, g, b2, cs) - infos[0].marginal_err) <= 1e-3 * infos[0].marginal_err + 2e-6


def test_cluster_equals_grid_kernel(env):
    """Both 2D solvers on the same batch: the same iteration counts and W1
    within the FP32 tolerance of each other."""
    probs = []
    for i, (ns, nf, eps) in enumerate([(48, 48, 0.02), (120, 90, 5e-3), (33, 511, 5e-3)]):
        a2, b2 = _rand2d(40 + i, ns, nf)
        probs.append((a2, b2, (1.0 / nf, 1.0 / ns), eps, 1e-5, 400))
    wc, ic, _ = _solve(env, probs)
    wg, ig, _ = _solve(env, probs, grid2d=True)
    for k in range(len(probs)):
        assert ic[k].team_size > 0 and ig[k].team_size == 0
        assert abs(ic[k].iters - ig[k].iters) <= 1
        assert abs(wc[k] - wg[k]) <= TOL32 * abs(wg[k])


def test_cluster_stop_rule_and_mixed_batch(env):
    """A batch mixing images the cluster kernel holds with one it does not
    (a 600-point row): every image stops within one iteration of the oracle's
    own stop and matches the oracle at the GPU's iteration count."""
    _, fs1 = env
    shapes = [(64, 80, 0.03), (20, 600, 0.05), (130, 70, 0.02), (9, 500, 0.05)]
    probs = []
    for i, (ns, nf, eps) in enumerate(shapes):
        a2, b2 = _rand2d(300 + i, ns, nf)
        probs.append((a2, b2, (1.0 / nf, 1.0 / ns), eps, 1e-5, 3000))
    w, infos, _ = _solve(env, probs)
    assert [i.team_size > 0 for i in infos] == [True, False, True, True]
    for (a2, b2, h, eps, tol, itr), info, wi in zip(probs, infos, w):
        assert info.status == fs1.FS1_OK and info.marginal_err <= tol
        _check_oracle(wi, info, a2, b2, h, eps, info.iters)
        ro = cref.solve(a2, b2, h, eps, tol, itr, tau=1e10)
        assert abs(ro.iters - info.iters) <= 1


def test_cluster_warm_start_resume_bit_identical(env):
    torch, fs1 = env
    ns, nf, eps = 70, 90, 5e-3
    a2, b2 = _rand2d(77, ns, nf)
    h = (1.0 / nf, 1.0 / ns)
    w_full, i_full, _ = _solve(env, [(a2, b2, h, eps, 0.0, 50)])
    _, _, pots = _solve(env, [(a2, b2, h, eps, 0.0, 20)], outs=True)
    w_res, i_res, _ = _solve(env, [(a2, b2, h, eps, 0.0, 30)], inits=[pots[0]])
    assert i_res[0].team_size > 0 and i_res[0].iters == 30
    assert w_res[0] == w_full[0]
    assert i_res[0].marginal_err == i_full[0].marginal_err


def test_cluster_no_iterations_and_invalid(env):
    """itr_max = 0 returns the initial iterate's cost and error; an image with
    a negative entry is refused without being solved."""
    _, fs1 = env
    ns, nf, eps = 40, 50, 0.02
    a2, b2 = _rand2d(9, ns, nf)
    bad = a2.copy()
    bad[3, 4] = -1e-3
    bad[3, 5] += 1e-3
    h = (1.0 / nf, 1.0 / ns)
    w, infos, _ = _solve(env, [(a2, b2, h, eps, 0.0, 0), (bad, b2, h, eps, 0.0, 10)])
    assert infos[0].iters == 0 and infos[0].status == fs1.FS1_ENOTCONV
    _check_oracle(w[0], infos[0], a2, b2, h, eps, 0)
    assert infos[1].status == fs1.FS1_EINVAL


def test_cluster_full_workload4_images(env):
    """Workload 4 (512 x 512 blobs, eps = 1e-3) for 40 iterations: four
    images, oracle at equal iteration count."""
    ps = [inputs.workload4(i, itr_max=40) for i in (2, 3, 4, 5)]
    probs = [(p.a, p.b, tuple(p.h), p.eps, 0.0, 40) for p in ps]
    w, infos, _ = _solve(env, probs)
    refs = cref.solve_many(probs, tau=1e10)
    for i, r in enumerate(refs):
        assert infos[i].team_size == 16   # 512 rows: 32 per CTA
        assert infos[i].iters == r.iters == 40
        assert abs(w[i] - r.w) <= TOL32 * abs(r.w)
        assert abs(infos[i].marginal_err - r.err) <= 1e-3 * r.err


def test_cluster_blob_images_at_c_near_8(env):
    """Blob images over a 1e-7 floor (the 2D benchmark's generator) at
    c = h / eps = 7.8, the largest c the cluster kernel takes: the scalings
    span hundreds of binary orders within a few points.  300 iterations stay on
    the cluster kernel (no fall-back to the grid kernel) and agree with the
    grid kernel: W, the marginal error, and the potentials point by point."""
    import numpy as np
    from paper_2202_10042_gb300 import inputs
    ps = [inputs.workload4(i, side=256, eps=(1.0 / 256) / 7.8) for i in range(2)]
    probs = [(p.a, p.b, tuple(p.h), p.eps, 0.0, 300) for p in ps]
    wc, ic, pc = _solve(env, probs, outs=True)
    wg, ig, pg = _solve(env, probs, grid2d=True, outs=True)
    for k in range(len(probs)):
        assert ic[k].team_size > 0 and ig[k].team_size == 0
        assert ic[k].iters == ig[k].iters == 300
        assert abs(wc[k] - wg[k]) <= TOL32 * abs(wg[k])
        assert abs(ic[k].marginal_err - ig[k].marginal_err) <= 1e-3 * ig[k].marginal_err
        (fc, gc), (fg, gg) = [(f.cpu().numpy(), g.cpu().numpy()) for f, g in (pc[k], pg[k])]
        assert np.max(np.abs(fc - fg)) <= 1e-3 and np.max(np.abs(gc - gg)) <= 1e-3
