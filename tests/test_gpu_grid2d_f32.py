"""The grid kernel's FP32 block-frame path against the CPU FP64 oracle: 2D
images whose lane chunks of P points span at most 64 nats (P h / eps <= 64)
on every axis of more than one point, where the general path would scan an
axis point by point in extended range (P' h / eps > 40 for its own P');
values FP32 with one power-of-two frame per block of 8 points.  These are
images with sides above 512 (beyond the cluster kernel) and h / eps of about
1.3 to 2.

Tolerances: relative W1 <= 1e-4 and marginal error within 1e-3 relative of the
oracle (FP32 stabilised), at the GPU's iteration count."""
import math

import numpy as np
import pytest

from oracle import cref, marginals

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


def _general_lanes(n, c):
    """Lanes per line of the general path (the fewest of 8, 16, 32 keeping at
    most 16 points per lane and its FP32-frame scan where 32 lanes allow it)."""
    frame32 = c * math.ceil(n / 32) <= 40
    for g in (8, 16):
        p = math.ceil(n / g)
        if p <= 16 and (not frame32 or c * p <= 40):
            return g
    return 32


def _f32_path(ns, nf, eps):
    """The rule of solve2d_f32_ok, restated."""
    per_point = False
    for n, h in ((nf, 1.0 / nf), (ns, 1.0 / ns)):
        if n < 2:
            continue
        c = h / eps
        g = 8 if n <= 128 else (16 if n <= 256 else 32)
        if c * math.ceil(math.ceil(n / g) / 8) * 8 > 64:
            return False
        per_point = per_point or c * math.ceil(n / _general_lanes(n, c)) > 40
    return per_point


def _solve(env, probs, outs=False, dtype=None):
    torch, fs1 = env
    s = fs1.Solver("log", "fp32")
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


def _check(w, info, a2, b2, h, eps, itr):
    ref = cref.solve(a2, b2, h, eps, 0.0, itr, tau=1e10)
    assert info.iters == ref.iters
    assert abs(w - ref.w) <= TOL32 * abs(ref.w), (w, ref.w)
    assert abs(info.marginal_err - ref.err) <= 1e-3 * ref.err + 1e-7, (info.marginal_err, ref.err)


# 32 lanes of 24 or 32 points, padded rows (nf not a multiple of 8), partial
# blocks and partly empty lanes, a single row and a single column
@pytest.mark.parametrize("ns,nf,eps", [
    (1024, 1024, 6e-4), (800, 800, 7e-4), (700, 900, 6e-4), (600, 777, 7e-4), (1, 900, 6e-4),
    (900, 1, 6e-4), (640, 640, 7e-4), (1000, 1000, 7e-4),
])
def test_f32_grid_against_oracle(env, ns, nf, eps):
    assert _f32_path(ns, nf, eps)
    a2, b2 = _rand2d(ns * 131 + nf, ns, nf)
    h = (1.0 / nf, 1.0 / ns)
    itr = 20
    w, infos, _ = _solve(env, [(a2, b2, h, eps, 0.0, itr)])
    _, fs1 = env
    assert infos[0].team_size == 0 and infos[0].status in (fs1.FS1_OK, fs1.FS1_ENOTCONV)
    _check(w[0], infos[0], a2, b2, h, eps, itr)


def test_f32_grid_potentials_and_marginals(env):
    """Potentials out, entry by entry, and the exact row marginal of the
    returned iterate."""
    ns, nf, eps, itr = 700, 900, 6e-4, 15
    assert _f32_path(ns, nf, eps)
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
    """One call with images of the FP32 path and images of the general path
    (its frame scans, and c P beyond 64): two grid launches; every image stops
    within one iteration of the oracle's own stop (or both reach the cap) and
    matches the oracle at the GPU's iteration count."""
    _, fs1 = env
    shapes = [(1, 900, 6e-4), (640, 640, 7e-4), (900, 1, 6e-4), (700, 600, 1.5e-3), (520, 40, 3e-4)]
    assert [_f32_path(*sh) for sh in shapes] == [True, True, True, False, False]
    probs = []
    for i, (ns, nf, eps) in enumerate(shapes):
        a2, b2 = _rand2d(500 + i, ns, nf)
        probs.append((a2, b2, (1.0 / nf, 1.0 / ns), eps, 1e-4, 300))
    w, infos, _ = _solve(env, probs)
    for (a2, b2, h, eps, tol, itr), info, wi in zip(probs, infos, w):
        assert info.team_size == 0 and info.status in (fs1.FS1_OK, fs1.FS1_ENOTCONV)
        assert (info.status == fs1.FS1_OK) == (info.marginal_err <= tol)
        _check(wi, info, a2, b2, h, eps, info.iters)
        ro = cref.solve(a2, b2, h, eps, tol, itr, tau=1e10)
        assert abs(ro.iters - info.iters) <= 1


def test_f32_grid_float32_inputs_batch(env):
    """Four images of a serving-size batch from float32 arrays, 8 iterations."""
    torch, _ = env
    probs = []
    for i, (side, eps) in enumerate(((1024, 6e-4), (800, 7e-4), (640, 7e-4), (700, 8e-4))):
        a2, b2 = _rand2d(70 + i, side, side)
        assert _f32_path(side, side, eps) or side == 700
        probs.append((a2, b2, (1.0 / side, 1.0 / side), eps, 0.0, 8))
    w, infos, _ = _solve(env, probs, dtype=torch.float32)
    refs = cref.solve_many([(a2.astype(np.float32).astype(np.float64), b2.astype(np.float32).astype(np.float64),
                             h, eps, 0.0, 8) for a2, b2, h, eps, tol, itr in probs], tau=1e10)
    for k, r in enumerate(refs):
        assert infos[k].team_size == 0 and infos[k].iters == 8
        assert abs(w[k] - r.w) <= TOL32 * abs(r.w), (k, w[k], r.w)
