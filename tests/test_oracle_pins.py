"""Pins of the CPU oracle against facts that do not come from the oracle itself:
closed forms, brute-force LP, limits in eps, invariants, the paper's stability
bound and the paper's printed plan agreement.  No GPU."""
import math
import os

import numpy as np
import pytest

from oracle import cref, dense, exact, recurrence
from paper_2202_10042_gb300 import inputs

HERE = os.path.dirname(os.path.abspath(__file__))


def _rel(x, y):
    return abs(x - y) / max(abs(y), 1e-300)


# ---------------------------------------------------------------------------
# closed forms of W1
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n,seed", [(2, 0), (3, 1), (5, 2), (8, 3), (8, 4)])
def test_exact_w1_cdf_equals_lp(n, seed):
    """The CDF formula and the brute-force LP are two independent routes to W1."""
    a, b = inputs.random_pair_1d(100 + seed, n, zeros=1 if seed % 2 else 0)
    h = 0.37
    lp = exact.w1_lp(a, b, dense.ground_cost_1d(n, h))
    assert abs(exact.w1_exact_1d(a, b, h) - lp) <= 1e-12


def test_exact_w1_hand_values():
    # unit mass moved 3 cells: W1 = 3h
    a = np.array([1.0, 0, 0, 0])
    b = np.array([0, 0, 0, 1.0])
    assert exact.w1_exact_1d(a, b, 0.5) == pytest.approx(1.5, abs=1e-15)
    # half the mass moved by one cell
    a = np.array([0.5, 0.5, 0.0])
    b = np.array([0.0, 0.5, 0.5])
    assert exact.w1_exact_1d(a, b, 1.0) == pytest.approx(1.0, abs=1e-15)


def test_lp_2d_small_grid():
    """2D L1 cost on a 2 x 4 grid: the entropic value approaches the LP as eps -> 0."""
    rng = np.random.default_rng(7)
    a2 = rng.uniform(0.1, 1, (2, 4)); a2 /= a2.sum()
    b2 = rng.uniform(0.1, 1, (2, 4)); b2 /= b2.sum()
    hf, hs = 0.25, 0.5
    C = dense.ground_cost_2d(4, 2, hf, hs)
    lp = exact.w1_lp(a2.reshape(-1), b2.reshape(-1), C)
    r = dense.solve_2d(a2, b2, hf, hs, 0.01, 1e-13, 200000, log=True)
    H = min(exact.entropy(a2), exact.entropy(b2))
    gap = r.w - lp
    assert -1e-9 <= gap <= 0.01 * H + 1e-9


# ---------------------------------------------------------------------------
# the dense Sinkhorn oracle
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("k", [1, 2, 4])
def test_entropic_gap_bound(k):
    """At convergence 0 <= <P_eps, C> - W1 <= eps * min(H(a), H(b)) (optimality
    of P_eps for <.,C> - eps H and H(a), H(b) <= H(P))."""
    n = 64
    h = 1.0 / n
    eps = h / k
    a, b = inputs.random_pair_1d(2, n, floor=0.05)
    W1 = exact.w1_exact_1d(a, b, h)
    r = dense.solve_1d(a, b, h, eps, 1e-11, 200000, log=True)
    assert r.err <= 1e-11
    slack = (n - 1) * h * r.err
    gap = r.w - W1
    assert -slack <= gap <= eps * min(exact.entropy(a), exact.entropy(b)) + slack


def test_eps_to_infinity_independent_coupling():
    """eps -> inf: K -> all ones, one iteration gives P = a b^T, so the return
    value is sum_ij a_i b_j |i-j| h."""
    n = 40
    h = 1.0 / n
    a, b = inputs.random_pair_1d(5, n, zeros=2)
    r = dense.solve_1d(a, b, h, 1e12, 0.0, 1)
    ref = float(a @ dense.ground_cost_1d(n, h) @ b)
    assert _rel(r.w, ref) < 1e-9


def test_eps_to_zero_diagonal_kernel():
    """eps << h: K -> identity, so P is diagonal, the cost is 0 and the
    column-marginal error is sum |a - b|."""
    n = 30
    a, b = inputs.random_pair_1d(6, n, floor=0.1)
    h = 1.0 / n
    r = dense.solve_1d(a, b, h, h / 1000.0, 0.0, 3)
    assert r.w == pytest.approx(0.0, abs=1e-300)
    assert r.err == pytest.approx(np.abs(a - b).sum(), rel=1e-12)


def test_row_marginal_exact_and_err_consistent():
    n = 100
    h = 1.0 / n
    a, b = inputs.random_pair_1d(8, n, floor=0.01)
    K = dense.gibbs_kernel_1d(n, h, 0.05)
    r = dense.sinkhorn_dense(a, b, K, dense.ground_cost_1d(n, h), 0.0, 37)
    P = dense.transport_plan(r.u, r.v, K)
    assert np.abs(P.sum(axis=1) - a).max() <= 1e-14
    assert abs(np.abs(P.sum(axis=0) - b).sum() - r.err) <= 1e-14


def test_reflection_invariance():
    """K is persymmetric: reversing both histograms reverses the iterates and
    leaves the cost unchanged at every l."""
    n = 77
    h = 1.0 / n
    a, b = inputs.random_pair_1d(9, n, zeros=1)
    for it in (0, 1, 5, 40):
        r1 = dense.solve_1d(a, b, h, 0.03, 0.0, it)
        r2 = dense.solve_1d(a[::-1], b[::-1], h, 0.03, 0.0, it)
        assert _rel(r1.w, r2.w) < 1e-12
        assert np.allclose(r1.u, r2.u[::-1], rtol=1e-12, atol=0)


def test_symmetry_at_convergence():
    n = 50
    h = 1.0 / n
    a, b = inputs.random_pair_1d(10, n, floor=0.05)
    r1 = dense.solve_1d(a, b, h, 0.05, 1e-13, 100000, log=True)
    r2 = dense.solve_1d(b, a, h, 0.05, 1e-13, 100000, log=True)
    assert _rel(r1.w, r2.w) < 1e-10


def test_log_twin_equals_plain():
    p = inputs.workload1(0, n=300)
    r1 = dense.solve_1d(p.a, p.b, p.h[0], p.eps, 0.0, 200)
    r2 = dense.solve_1d(p.a, p.b, p.h[0], p.eps, 0.0, 200, log=True)
    assert r1.iters == r2.iters == 200
    assert _rel(r1.w, r2.w) < 1e-12
    assert np.allclose(np.log(r1.u), r2.f, rtol=0, atol=1e-10)


def test_single_point():
    r = dense.solve_1d(np.array([1.0]), np.array([1.0]), 0.1, 0.01, 0.0, 5)
    assert r.w == 0.0 and r.err == pytest.approx(0.0, abs=1e-15)


def test_2d_product_factorisation():
    """For a = a_y (x) a_x, b = b_y (x) b_x the separable kernel keeps the
    iterates in product form at every l (u = u_y (x) u_x), so the plan is
    P_y (x) P_x and W_2D = m_y W_x + m_x W_y with m the 1D plan masses; after
    the first u-update every plan has mass 1 and W_2D = W_x + W_y."""
    a2, b2, (ax, bx), (ay, by) = inputs.product_pair_2d(0, 11, 6)
    hf, hs, eps = 1 / 11, 1 / 6, 0.08
    Kx = dense.gibbs_kernel_1d(11, hf, eps)
    Ky = dense.gibbs_kernel_1d(6, hs, eps)
    for it in (0, 1, 3, 12):
        r2 = dense.solve_2d(a2, b2, hf, hs, eps, 0.0, it)
        rx = dense.solve_1d(ax, bx, hf, eps, 0.0, it)
        ry = dense.solve_1d(ay, by, hs, eps, 0.0, it)
        assert np.allclose(r2.u.reshape(6, 11), np.outer(ry.u, rx.u), rtol=1e-12, atol=0)
        mx = float(rx.u @ Kx @ rx.v)
        my = float(ry.u @ Ky @ ry.v)
        assert _rel(r2.w, my * rx.w + mx * ry.w) < 1e-12
        if it >= 1:
            assert _rel(r2.w, rx.w + ry.w) < 1e-12


def test_2d_single_row_is_1d():
    n = 25
    a, b = inputs.random_pair_1d(11, n, floor=0.01)
    r2 = dense.solve_2d(a[None, :], b[None, :], 1 / n, 0.3, 0.04, 0.0, 30)
    r1 = dense.solve_1d(a, b, 1 / n, 0.04, 0.0, 30)
    assert _rel(r2.w, r1.w) < 1e-13 and r2.iters == r1.iters


# ---------------------------------------------------------------------------
# the recurrences (Section 3 / 4)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n", [1, 2, 3, 37, 256])
def test_horner_equals_dense_matvec(n):
    rng = np.random.default_rng(n)
    x = rng.uniform(0, 1, n)
    for lam in (0.0, 1e-3, 0.5, 0.95, 1.0):
        K = lam ** np.abs(np.arange(n)[:, None] - np.arange(n)[None, :]) if lam > 0 else np.eye(n)
        p, q = recurrence.horner_matvec(x, lam)
        assert np.allclose(p + q, K @ x, rtol=1e-13, atol=0)
        # lower part and strict upper part separately (eq. "meshpoly")
        assert np.allclose(p, np.tril(K) @ x, rtol=1e-13, atol=0)


def test_stability_bound():
    """Section 3: |(p+q)^1_k - (p+q)^2_k| <= ((2 - (lam^k + lam^{N-k+1}))/(1-lam) - 1) delta
    for inputs that differ by at most delta (k 1-based)."""
    n, lam, delta = 60, 0.9, 1e-3
    rng = np.random.default_rng(1)
    x1 = rng.uniform(0, 1, n)
    for trial in range(5):
        d = rng.uniform(-delta, delta, n)
        if trial == 0:
            d[:] = delta          # the bound is attained by a constant shift
        p1, q1 = recurrence.horner_matvec(x1, lam)
        p2, q2 = recurrence.horner_matvec(x1 + d, lam)
        k = np.arange(1, n + 1)
        bound = ((2 - (lam ** k + lam ** (n - k + 1))) / (1 - lam) - 1) * delta
        dev = np.abs((p1 + q1) - (p2 + q2))
        assert np.all(dev <= bound * (1 + 1e-9))
        if trial == 0:
            assert np.allclose(dev, bound, rtol=1e-9)


@pytest.mark.parametrize("n", [1, 2, 45])
def test_distance_weighted_matvec(n):
    rng = np.random.default_rng(3)
    x = rng.uniform(0, 1, n)
    lam = 0.8
    D = np.abs(np.arange(n)[:, None] - np.arange(n)[None, :]).astype(float)
    assert np.allclose(recurrence.distance_matvec(x, lam), (lam ** D * D) @ x, rtol=1e-13, atol=1e-300)


def test_lse_recurrence():
    rng = np.random.default_rng(4)
    n, c = 40, 0.7
    f = rng.normal(0, 5, n)
    f[7] = -np.inf
    R, S = recurrence.lse_matvec(f, c)
    K = np.exp(-c * np.abs(np.arange(n)[:, None] - np.arange(n)[None, :]))
    assert np.allclose(np.logaddexp(R, S), np.log(K @ np.exp(f)), rtol=0, atol=1e-12)


@pytest.mark.parametrize("n", [1, 2, 45])
def test_lse_distance_matvec_against_linear_and_brute_force(n):
    """The log-domain distance-weighted product equals log of distance_matvec
    and of the O(N^2) definition where e^g is representable."""
    rng = np.random.default_rng(5 + n)
    g = rng.normal(0, 3, n)
    c = 0.35
    D = np.abs(np.arange(n)[:, None] - np.arange(n)[None, :]).astype(float)
    brute = (np.exp(-c * D) * D) @ np.exp(g)
    got = recurrence.lse_distance_matvec(g, c)
    lin = recurrence.distance_matvec(np.exp(g), math.exp(-c))
    if n == 1:
        assert got[0] == -np.inf and brute[0] == 0.0
        return
    assert np.allclose(got, np.log(brute), rtol=0, atol=1e-12)
    assert np.allclose(got, np.log(lin), rtol=0, atol=1e-12)


def test_lse_distance_matvec_large_potentials_and_zeros():
    """Potentials of magnitude 1e4 (e^g far outside FP64) and zero entries:
    against the O(N^2) definition taken in log space term by term,
    log sum_j exp(g_j - c |k-j| + log |k-j|)."""
    rng = np.random.default_rng(6)
    n, c = 60, 2.5
    g = np.cumsum(rng.uniform(-2 * c, 2 * c, n)) + 1e4
    g[[4, 33]] = -np.inf
    got = recurrence.lse_distance_matvec(g, c)
    for k in range(n):
        terms = [g[j] - c * abs(k - j) + math.log(abs(k - j)) for j in range(n) if j != k and g[j] > -np.inf]
        m = max(terms)
        ref = m + math.log(sum(math.exp(t - m) for t in terms))
        assert abs(got[k] - ref) <= 1e-12 * abs(ref)


def test_fs1_equals_dense_sinkhorn():
    p = inputs.workload1(3, n=128)
    h = p.h[0]
    rd = dense.solve_1d(p.a, p.b, h, p.eps, 0.0, 60)
    for r in (recurrence.fs1_plain(p.a, p.b, h, p.eps, 0.0, 60),
              recurrence.fs1_log(p.a, p.b, h, p.eps, 0.0, 60),
              recurrence.fs1_stabilised(p.a, p.b, h, p.eps, 0.0, 60, tau=1e3)):
        assert r.iters == rd.iters
        assert _rel(r.w, rd.w) < 1e-11
        assert abs(r.err - rd.err) <= 1e-9 * rd.err + 1e-14


def test_fs1_2d_equals_dense():
    rng = np.random.default_rng(12)
    a2 = rng.uniform(0, 1, (5, 8)); a2 /= a2.sum()
    b2 = rng.uniform(0, 1, (5, 8)); b2 /= b2.sum()
    hf, hs, eps = 1 / 8, 1 / 5, 0.1
    rd = dense.solve_2d(a2, b2, hf, hs, eps, 0.0, 25)
    rr = recurrence.fs1_plain_2d(a2, b2, hf, hs, eps, 0.0, 25)
    assert _rel(rr.w, rd.w) < 1e-12 and _rel(rr.err, rd.err) < 1e-9
    x = rng.uniform(0, 1, (5, 8))
    K = dense.gibbs_kernel_2d(8, 5, hf, hs, eps)
    got = recurrence.horner_matvec_2d(x, math.exp(-hf / eps), math.exp(-hs / eps))
    assert np.allclose(got.reshape(-1), K @ x.reshape(-1), rtol=1e-13, atol=0)


def test_plan_agreement_magnitude_table1():
    """Table 1 prints ||P_FS1 - P||_F at round-off (6.54e-15 at N = 500).
    Same workload shape: grid on [-3, 3], dx = 6/(N-1), U[0,1] weights
    normalised, eps = 1e-3, 1000 iterations (Section 5.1)."""
    rows = [l.split() for l in open(os.path.join(HERE, "golden", "paper_plan_agreement.txt"))
            if l.strip() and not l.startswith("#")]
    printed = {int(r[2]): float(r[5]) for r in rows if r[1] == "random_1d"}
    n = 500
    dx = 6.0 / (n - 1)
    a, b = inputs.random_pair_1d(500, n)
    eps = 1e-3
    K = dense.gibbs_kernel_1d(n, dx, eps)
    rd = dense.sinkhorn_dense(a, b, K, dense.ground_cost_1d(n, dx), 0.0, 1000)
    rr = recurrence.fs1_plain(a, b, dx, eps, 0.0, 1000)
    diff = np.linalg.norm(dense.transport_plan(rd.u, rd.v, K) - dense.transport_plan(rr.u, rr.v, K))
    assert diff <= max(100 * printed[n], 1e-13)


# ---------------------------------------------------------------------------
# the C oracle
# ---------------------------------------------------------------------------

def test_cref_matvec_1d_2d():
    rng = np.random.default_rng(13)
    for n in (1, 2, 63):
        x = rng.uniform(0, 1, n)
        K = dense.gibbs_kernel_1d(n, 1 / 64, 0.05)
        assert np.allclose(cref.matvec(x, 1 / 64, 0.05), K @ x, rtol=1e-13, atol=0)
        D = dense.ground_cost_1d(n, 1.0)
        assert np.allclose(cref.matvec(x, 1 / 64, 0.05, weighted_fast=True), (K * D) @ x,
                           rtol=1e-12, atol=1e-300)
    x2 = rng.uniform(0, 1, (6, 9))
    K2 = dense.gibbs_kernel_2d(9, 6, 0.1, 0.2, 0.3)
    assert np.allclose(cref.matvec(x2, (0.1, 0.2), 0.3).reshape(-1), K2 @ x2.reshape(-1), rtol=1e-13)
    Cf = dense.ground_cost_2d(9, 6, 1.0, 0.0)
    Cs = dense.ground_cost_2d(9, 6, 0.0, 1.0)
    assert np.allclose(cref.matvec(x2, (0.1, 0.2), 0.3, weighted_fast=True).reshape(-1),
                       (K2 * Cf) @ x2.reshape(-1), rtol=1e-12)
    assert np.allclose(cref.matvec(x2, (0.1, 0.2), 0.3, weighted_slow=True).reshape(-1),
                       (K2 * Cs) @ x2.reshape(-1), rtol=1e-12)


@pytest.mark.parametrize("tau", [math.inf, 1e10, 1e3])
def test_cref_1d_equals_dense(tau):
    p = inputs.workload1(1, n=400)
    h = p.h[0]
    rd = dense.solve_1d(p.a, p.b, h, p.eps, 0.0, 150, log=True)
    rc = cref.solve(p.a, p.b, h, p.eps, 0.0, 150, tau=tau, potentials=True)
    assert rc.status == cref.OK and rc.iters == rd.iters
    assert _rel(rc.w, rd.w) < 1e-11
    assert abs(rc.err - rd.err) <= 1e-8 * rd.err + 1e-13
    assert np.allclose(rc.f - rc.f[0], rd.f - rd.f[0], rtol=0, atol=1e-8)


def test_cref_stopping_rule():
    p = inputs.workload1(2, n=200)
    h = p.h[0]
    for tol in (1e-2, 1e-5, 1e-9):
        rd = dense.solve_1d(p.a, p.b, h, p.eps, tol, 100000)
        rc = cref.solve(p.a, p.b, h, p.eps, tol, 100000, tau=1e10)
        assert rc.iters == rd.iters and rc.err <= tol and _rel(rc.w, rd.w) < 1e-10


def test_cref_small_eps_stabilised():
    """A small-eps case where the stabilised form must carry the iteration."""
    n = 300
    h = 1.0 / n
    a, b = inputs.random_pair_1d(14, n, floor=0.02)
    eps = h / 3
    rd = dense.solve_1d(a, b, h, eps, 0.0, 400, log=True)
    for tau in (1e3, 1e10):
        rc = cref.solve(a, b, h, eps, 0.0, 400, tau=tau)
        assert rc.status == cref.OK and _rel(rc.w, rd.w) < 1e-9


def test_cref_abnormal_termination():
    """Section 5.2: without stabilisation the iteration terminates abnormally at
    small eps; with it, it does not."""
    n = 1000
    x = (np.arange(n) + 0.5) / n
    a = np.exp(-0.5 * ((x - 0.2) / 0.03) ** 2) + 1e-3; a /= a.sum()
    b = np.exp(-0.5 * ((x - 0.8) / 0.03) ** 2) + 1e-3; b /= b.sum()
    r = cref.solve(a, b, 1 / n, 5e-4, 1e-9, 3000, tau=math.inf)
    s = cref.solve(a, b, 1 / n, 5e-4, 1e-9, 3000, tau=1e10)
    assert r.status == cref.ENUMERIC and 0 < r.iters < 3000
    assert s.status == cref.OK and math.isfinite(s.w)


def test_cref_2d_equals_dense_and_product():
    a2, b2, (ax, bx), (ay, by) = inputs.product_pair_2d(1, 10, 7)
    hf, hs, eps = 0.1, 1 / 7, 0.05
    rd = dense.solve_2d(a2, b2, hf, hs, eps, 0.0, 40, log=True)
    for tau in (math.inf, 10.0):
        rc = cref.solve(a2, b2, (hf, hs), eps, 0.0, 40, tau=tau)
        assert rc.status == cref.OK and rc.iters == 40 and _rel(rc.w, rd.w) < 1e-11
    rx = cref.solve(ax, bx, hf, eps, 0.0, 40, tau=math.inf)
    ry = cref.solve(ay, by, hs, eps, 0.0, 40, tau=math.inf)
    assert _rel(rd.w, rx.w + ry.w) < 1e-12


def test_cref_workload1_full():
    """Workload 1 at its full size (N = 1000, 1000 iterations): C oracle equals
    the dense definition and stays above the exact W1 minus the marginal slack."""
    p = inputs.workload1(0)
    h = p.h[0]
    rd = dense.solve_1d(p.a, p.b, h, p.eps, p.tol, p.itr_max)
    rc = cref.solve(p.a, p.b, h, p.eps, p.tol, p.itr_max, tau=math.inf)
    assert rc.iters == rd.iters == 1000
    assert _rel(rc.w, rd.w) < 1e-12
    W1 = exact.w1_exact_1d(p.a, p.b, h)
    assert rc.w >= W1 - (p.a.size - 1) * h * rc.err - 1e-12


# ---------------------------------------------------------------------------
# 3D: the extension to a third axis stated by Section 4's closing remark
# ---------------------------------------------------------------------------

def test_3d_ground_cost_and_kernel_structure():
    """The 3D cost is the sum of the axis distances (brute force over the
    coordinates of the fast-first flattening) and K = exp(-C / eps) is the
    Kronecker product of the three 1D kernels."""
    nf, nm, ns, h = 3, 4, 2, (0.1, 0.2, 0.3)
    C = dense.ground_cost_3d(nf, nm, ns, *h)
    pts = [(i, j, k) for k in range(ns) for j in range(nm) for i in range(nf)]
    for p, (i1, j1, k1) in enumerate(pts):
        for q, (i2, j2, k2) in enumerate(pts):
            assert C[p, q] == pytest.approx(abs(i1 - i2) * h[0] + abs(j1 - j2) * h[1] + abs(k1 - k2) * h[2],
                                            abs=1e-15)
    assert np.allclose(np.exp(-C / 0.7), dense.gibbs_kernel_3d(nf, nm, ns, *h, 0.7), rtol=1e-13, atol=0)


def test_lp_3d_small_grid():
    """3D L1 cost on a 3 x 2 x 2 grid: the entropic value approaches the LP."""
    rng = np.random.default_rng(17)
    a3 = rng.uniform(0.1, 1, (2, 2, 3)); a3 /= a3.sum()
    b3 = rng.uniform(0.1, 1, (2, 2, 3)); b3 /= b3.sum()
    h = (1 / 3, 0.5, 0.5)
    C = dense.ground_cost_3d(3, 2, 2, *h)
    lp = exact.w1_lp(a3.reshape(-1), b3.reshape(-1), C)
    r = dense.solve_3d(a3, b3, h, 0.01, 1e-13, 200000, log=True)
    H = min(exact.entropy(a3), exact.entropy(b3))
    gap = r.w - lp
    assert -1e-9 <= gap <= 0.01 * H + 1e-9


def test_3d_product_factorisation():
    """Separable inputs keep the iterates in product form at every l, so
    W_3D = m_y m_z W_x + m_x m_z W_y + m_x m_y W_z with m the 1D plan masses;
    after the first u-update every mass is 1."""
    a3, b3, ((ax, bx), (ay, by), (az, bz)) = inputs.product_pair_3d(0, 7, 5, 4)
    h, eps = (1 / 7, 1 / 5, 1 / 4), 0.1
    Ks = [dense.gibbs_kernel_1d(n, hh, eps) for n, hh in zip((7, 5, 4), h)]
    for it in (0, 1, 3, 10):
        r3 = dense.solve_3d(a3, b3, h, eps, 0.0, it)
        rs = [dense.solve_1d(p, q, hh, eps, 0.0, it) for (p, q), hh in zip(((ax, bx), (ay, by), (az, bz)), h)]
        u = np.einsum("k,j,i->kji", rs[2].u, rs[1].u, rs[0].u)
        assert np.allclose(r3.u.reshape(4, 5, 7), u, rtol=1e-12, atol=0)
        m = [float(r.u @ K @ r.v) for r, K in zip(rs, Ks)]
        want = m[1] * m[2] * rs[0].w + m[0] * m[2] * rs[1].w + m[0] * m[1] * rs[2].w
        assert _rel(r3.w, want) < 1e-12
        if it >= 1:
            assert _rel(r3.w, rs[0].w + rs[1].w + rs[2].w) < 1e-12


def test_3d_single_slab_is_2d():
    rng = np.random.default_rng(19)
    a2 = rng.uniform(0.05, 1, (5, 6)); a2 /= a2.sum()
    b2 = rng.uniform(0.05, 1, (5, 6)); b2 /= b2.sum()
    r3 = dense.solve_3d(a2[None], b2[None], (1 / 6, 1 / 5, 0.7), 0.05, 0.0, 25)
    r2 = dense.solve_2d(a2, b2, 1 / 6, 1 / 5, 0.05, 0.0, 25)
    assert _rel(r3.w, r2.w) < 1e-13 and r3.iters == r2.iters


def test_cref_matvec_3d():
    rng = np.random.default_rng(23)
    x3 = rng.uniform(0, 1, (3, 4, 5))
    h, eps = (0.1, 0.2, 0.3), 0.25
    K3 = dense.gibbs_kernel_3d(5, 4, 3, *h, eps)
    assert np.allclose(cref.matvec(x3, h, eps).reshape(-1), K3 @ x3.reshape(-1), rtol=1e-13, atol=0)
    for ax in range(3):
        unit = [0.0, 0.0, 0.0]
        unit[ax] = 1.0
        D = dense.ground_cost_3d(5, 4, 3, *unit)
        got = cref.matvec(x3, h, eps, weighted_axes=1 << ax).reshape(-1)
        assert np.allclose(got, (K3 * D) @ x3.reshape(-1), rtol=1e-12, atol=1e-300)


@pytest.mark.parametrize("tau", [math.inf, 10.0])
def test_cref_3d_equals_dense(tau):
    rng = np.random.default_rng(29)
    a3 = rng.uniform(0.05, 1, (4, 5, 6)); a3 /= a3.sum()
    b3 = rng.uniform(0.05, 1, (4, 5, 6)); b3 /= b3.sum()
    h, eps = (1 / 6, 1 / 5, 1 / 4), 0.04
    rd = dense.solve_3d(a3, b3, h, eps, 0.0, 30, log=True)
    rc = cref.solve(a3, b3, h, eps, 0.0, 30, tau=tau)
    assert rc.status == cref.OK and rc.iters == rd.iters == 30
    assert _rel(rc.w, rd.w) < 1e-11
    assert abs(rc.err - rd.err) <= 1e-11 * max(1.0, rd.err)
    # the stop rule on the 3D marginal error
    rt = cref.solve(a3, b3, h, eps, 1e-6, 5000, tau=tau)
    rdt = dense.solve_3d(a3, b3, h, eps, 1e-6, 5000, log=True)
    assert rt.iters == rdt.iters and rt.err <= 1e-6


def test_cref_3d_product_equals_three_1d():
    a3, b3, ((ax, bx), (ay, by), (az, bz)) = inputs.product_pair_3d(1, 9, 6, 5)
    h, eps = (1 / 9, 1 / 6, 1 / 5), 0.05
    r3 = cref.solve(a3, b3, h, eps, 0.0, 40, tau=math.inf)
    r1 = [cref.solve(p, q, hh, eps, 0.0, 40, tau=math.inf)
          for (p, q), hh in zip(((ax, bx), (ay, by), (az, bz)), h)]
    assert _rel(r3.w, sum(r.w for r in r1)) < 1e-12
