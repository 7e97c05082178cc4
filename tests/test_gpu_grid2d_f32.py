"""The grid kernel's FP32 block-frame path (2D images whose lane chunks of P
points span at most 64 nats, P h / eps <= 64, on every axis of more than one
point; values FP32 with one power-of-two frame per block of 8 points) against
the CPU FP64 oracle, forced with fs1_config.grid2d = 1 for shapes the cluster
kernel would otherwise take, and by default for sides above 512.

Tolerances: relative W1 <= 1e-4 and marginal error within 1e-3 relative of the
oracle (FP32 stabilised), at the GPU's iteration count."""
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


def _solve(env, probs, grid2d=True, outs=False, dtype=None):
    torch, fs1 = env
    s = fs1.Solver("log", "fp32", grid2d=grid2d)
    keep, ps, pots = [], [], []
    for (a2, b2, h, eps, tol, itr) in probs:
        ta = torch.tensor(a2, dtype=dtype or torch.float64, device="cuda")
        tb = torch.tensor(b2, dtype=dtype or torch.float64, device="cuda")
        keep += [ta, tb]
        kw = {}
        if outs:
            f = torch.empty(a2.shape, dtype=torch.float64, device="cuda")
            g = torch.empty(a2.shape, dtype=torch.float64, device="cuda")
            pots.append((f, g))
            kw.update(f_out=f, g_out=g)
        ps.append(fs1.Solver.problem(ta, tb, h, eps, tol, itr, **kw))
    st, w, infos = s.solve(ps)
    s.close()
    return w, infos, pots


def _f32_path(ns, nf, eps):
    def p_of(n):
        g = 8 if n <= 128 else (16 if n <= 256 else 32)
        return -(-(-(-n // g)) // 8) * 8
    return (nf == 1 or p_of(nf) / nf / eps <= 64) and (ns == 1 or p_of(ns) / ns / eps <= 64)


def _check(w, info, a2, b2, h, eps, itr):
    ref = cref.solve(a2, b2, h, eps, 0.0, itr, tau=1e10)
    assert info.iters == ref.iters
    assert abs(w - ref.w) <= TOL32 * abs(ref.w), (w, ref.w)
    assert abs(info.marginal_err - ref.err) <= 1e-3 * ref.err + 1e-7, (info.marginal_err, ref.err)


# every lane geometry (8, 16, 32 lanes; 8 to 32 points per lane), ragged rows
# and columns (padded rows, partial blocks, partly empty lanes), single rows
# and columns, c P up to the limit of 64 nats
@pytest.mark.parametrize("ns,nf,eps", [
    (1, 37, 0.02), (29, 1, 0.02), (5, 3, 0.1), (9, 17, 0.03), (64, 64, 2e-3), (100, 129, 5e-3),
    (257, 200, 2e-3), (130, 700, 2e-3), (513, 300, 1e-3), (1000, 1000, 1e-3), (33, 1024, 0.04),
    (1024, 24, 6e-3), (600, 777, 1e-3),
])
def test_f32_grid_against_oracle(env, ns, nf, eps):
    a2, b2 = _rand2d(ns * 131 + nf, ns, nf)
    h = (1.0 / nf, 1.0 / ns)
    assert _f32_path(ns, nf, eps)
    itr = 25
    w, infos, _ = _solve(env, [(a2, b2, h, eps, 0.0, itr)])
    _, fs1 = env
    assert infos[0].team_size == 0 and infos[0].status in (fs1.FS1_OK, fs1.FS1_ENOTCONV)
    _check(w[0], infos[0], a2, b2, h, eps, itr)


def test_f32_grid_potentials_and_marginals(env):
    """Potentials out, entry by entry, and the exact row marginal of the
    returned iterate."""
    ns, nf, eps, itr = 300, 650, 1e-3, 20
    a2, b2 = _rand2d(12, ns, nf)
    h = (1.0 / nf, 1.0 / ns)
    w, infos, pots = _solve(env, [(a2, b2, h, eps, 0.0, itr)], outs=True)
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


def test_f32_grid_stop_rule_and_mixed_call(env):
    """One call with images of the FP32 path and images beyond it (c P > 64):
    two grid launches; every image stops within one iteration of the oracle's
    own stop and matches the oracle at the GPU's iteration count."""
    _, fs1 = env
    shapes = [(64, 80, 0.03), (20, 600, 0.05), (130, 70, 0.002), (700, 40, 0.02), (40, 100, 1e-3)]
    assert [_f32_path(*sh) for sh in shapes] == [True, True, False, True, False]
    probs = []
    for i, (ns, nf, eps) in enumerate(shapes):
        a2, b2 = _rand2d(500 + i, ns, nf)
        probs.append((a2, b2, (1.0 / nf, 1.0 / ns), eps, 1e-5, 3000))
    w, infos, _ = _solve(env, probs)
    for (a2, b2, h, eps, tol, itr), info, wi in zip(probs, infos, w):
        assert info.status in (fs1.FS1_OK, fs1.FS1_ENOTCONV)
        assert (info.status == fs1.FS1_OK) == (info.marginal_err <= tol)
        _check(wi, info, a2, b2, h, eps, info.iters)
        ro = cref.solve(a2, b2, h, eps, tol, itr, tau=1e10)
        assert abs(ro.iters - info.iters) <= 1
    assert sum(i.status == fs1.FS1_OK for i in infos) >= 3


def test_f32_grid_equals_cluster_kernel(env):
    """The grid kernel's FP32 path and the cluster kernel on the same images:
    the same iteration counts and W1 within the FP32 tolerance."""
    probs = []
    for i, (ns, nf, eps) in enumerate([(48, 48, 0.02), (120, 90, 5e-3), (512, 512, 1e-3)]):
        a2, b2 = _rand2d(40 + i, ns, nf)
        probs.append((a2, b2, (1.0 / nf, 1.0 / ns), eps, 1e-5, 300))
    wg, ig, _ = _solve(env, probs)
    wc, ic, _ = _solve(env, probs, grid2d=False)
    for k in range(len(probs)):
        assert ig[k].team_size == 0 and ic[k].team_size > 0
        assert abs(ic[k].iters - ig[k].iters) <= 1
        assert abs(wc[k] - wg[k]) <= TOL32 * abs(wc[k])


def test_f32_grid_big_images_by_default(env):
    """Sides above 512 (beyond the cluster kernel) take the FP32 grid path by
    default; float32 inputs; four images of a serving-size batch."""
    torch, _ = env
    probs = []
    for i, side in enumerate((600, 800, 1024, 700)):
        a2, b2 = _rand2d(70 + i, side, side)
        probs.append((a2, b2, (1.0 / side, 1.0 / side), 2e-3, 0.0, 8))
    w, infos, _ = _solve(env, probs, grid2d=False, dtype=torch.float32)
    refs = cref.solve_many([(a2.astype(np.float32).astype(np.float64), b2.astype(np.float32).astype(np.float64),
                             h, eps, 0.0, 8) for a2, b2, h, eps, tol, itr in probs], tau=1e10)
    for k, r in enumerate(refs):
        assert infos[k].team_size == 0 and infos[k].iters == 8
        assert abs(w[k] - r.w) <= TOL32 * abs(r.w), (k, w[k], r.w)
