"""Dense FP64 Sinkhorn: the plain definitions the FS-1 iteration must reproduce.

Test infrastructure only (see ``oracle/__init__.py``).

Notation: a, b are the two histograms (the paper's u, v of Section 2); u, v
are the Sinkhorn scalings (the paper's phi, psi); f = log u, g = log v are the
dimensionless log potentials.

Parity: pinned by tests/test_oracle_pins.py against the exact W1 (CDF), a
brute-force LP (1D, 2D and 3D grids), the entropic gap bound, marginal
invariants, and the 2D and 3D product factorisations.
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np
from scipy.special import logsumexp


@dataclasses.dataclass
class SinkhornResult:
    w: float          # transport cost <P, C> (the value Algorithm 1 returns)
    iters: int        # completed iterations l
    err: float        # marginal L1 error at the returned iterate
    u: Optional[np.ndarray] = None
    v: Optional[np.ndarray] = None
    f: Optional[np.ndarray] = None
    g: Optional[np.ndarray] = None
    status: int = 0   # 0 ok, 1 non-finite value met (abnormal termination)


# ---------------------------------------------------------------------------
# kernels and costs
# ---------------------------------------------------------------------------

def ground_cost_1d(n: int, h: float) -> np.ndarray:
    """C_ij = |i - j| h  (Section 2, discretised problem)."""
    i = np.arange(n, dtype=np.float64)
    return np.abs(i[:, None] - i[None, :]) * h


def gibbs_kernel_1d(n: int, h: float, eps: float) -> np.ndarray:
    """K_ij = exp(-|i - j| h / eps)  (Section 2, derivative of the Lagrangian)."""
    return np.exp(-ground_cost_1d(n, h) / eps)


def ground_cost_2d(n_fast: int, n_slow: int, h_fast: float, h_slow: float) -> np.ndarray:
    """Cost |i1 - i2| h1 + |j1 - j2| h2 on an n_fast x n_slow grid (Section 4,
    eq. "2d disc entropy problem").  Points are flattened with the first index
    (fast axis, spacing h1) running fastest, the paper's column-major order,
    which is numpy's C order of an (n_slow, n_fast) array."""
    cf = ground_cost_1d(n_fast, h_fast)
    cs = ground_cost_1d(n_slow, h_slow)
    return (cs[:, None, :, None] + cf[None, :, None, :]).reshape(n_fast * n_slow, n_fast * n_slow)


def gibbs_kernel_2d(n_fast: int, n_slow: int, h_fast: float, h_slow: float, eps: float) -> np.ndarray:
    """Block kernel of Section 4: K = [lambda_2^{|k-l|} K_0] with
    K_0 = [lambda_1^{|i-j|}], lambda_1 = exp(-h1/eps), lambda_2 = exp(-h2/eps)."""
    k0 = gibbs_kernel_1d(n_fast, h_fast, eps)
    k2 = gibbs_kernel_1d(n_slow, h_slow, eps)
    return np.kron(k2, k0)


def ground_cost_3d(n_fast: int, n_mid: int, n_slow: int, h_fast: float, h_mid: float,
                   h_slow: float) -> np.ndarray:
    """Cost |di| h1 + |dj| h2 + |dk| h3 on an n_fast x n_mid x n_slow grid: the
    L1 cost of Section 4 extended to a third axis (its closing remark).
    Points are flattened fast axis first, as numpy's C order of an
    (n_slow, n_mid, n_fast) array."""
    cf = ground_cost_1d(n_fast, h_fast)
    cm = ground_cost_1d(n_mid, h_mid)
    cs = ground_cost_1d(n_slow, h_slow)
    n = n_fast * n_mid * n_slow
    return (cs[:, None, None, :, None, None] + cm[None, :, None, None, :, None] +
            cf[None, None, :, None, None, :]).reshape(n, n)


def gibbs_kernel_3d(n_fast: int, n_mid: int, n_slow: int, h_fast: float, h_mid: float,
                    h_slow: float, eps: float) -> np.ndarray:
    """K = K_slow (x) K_mid (x) K_fast, the separable kernel of the 3D cost."""
    return np.kron(gibbs_kernel_1d(n_slow, h_slow, eps),
                   np.kron(gibbs_kernel_1d(n_mid, h_mid, eps), gibbs_kernel_1d(n_fast, h_fast, eps)))


# ---------------------------------------------------------------------------
# the Sinkhorn loop
# ---------------------------------------------------------------------------

def marginal_error(u, v, K, b) -> float:
    """|| diag(v) K^T u - b ||_1, the stopping quantity of Algorithm 1 (the
    while condition) and of Section 5's experiments."""
    return float(np.abs(v * (K.T @ u) - b).sum())


def transport_cost(u, v, K, C) -> float:
    """sum_ij u_i K_ij C_ij v_j: the value Algorithm 1 returns."""
    return float(u @ ((K * C) @ v))


def sinkhorn_dense(a, b, K, C, tol: float, itr_max: int) -> SinkhornResult:
    """Sinkhorn iteration eq. "update_sinkhorn" with a dense K, in the loop
    order of Algorithm 1: start from u = v = 1/N; while l < itr_max and the
    column-marginal error exceeds tol: v <- b / K^T u, u <- a / K v, l += 1.
    Returns the transport cost of the final (u, v)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    n = a.size
    u = np.full(n, 1.0 / n)
    v = np.full(n, 1.0 / n)
    ell = 0
    status = 0
    while True:
        ktu = K.T @ u
        err = float(np.abs(v * ktu - b).sum())
        if not np.isfinite(err):
            status = 1
            break
        if ell >= itr_max or err <= tol:
            break
        with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
            v = b / ktu
            u = a / (K @ v)
        ell += 1
    w = transport_cost(u, v, K, C) if status == 0 else float("nan")
    return SinkhornResult(w, ell, err, u=u, v=v, status=status)


def sinkhorn_dense_log(a, b, C, eps: float, tol: float, itr_max: int,
                       f0=None, g0=None) -> SinkhornResult:
    """Log-domain twin of sinkhorn_dense (the stabilisation of the Remark in
    Section 2 taken to its limit: every iterate fully absorbed into the
    potentials).  With f = log u, g = log v and M = -C / eps:
        g <- log b - logsumexp_i(f_i + M_ij)
        f <- log a - logsumexp_j(g_j + M_ij)
    which equals the plain update in exact arithmetic.  f = g = -log N at
    start (u = v = 1/N); zero mass gives -inf potentials."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    n = a.size
    M = -np.asarray(C, dtype=np.float64) / eps
    with np.errstate(divide="ignore"):
        la = np.log(a)
        lb = np.log(b)
    f = np.full(n, -np.log(n)) if f0 is None else np.array(f0, dtype=np.float64)
    g = np.full(n, -np.log(n)) if g0 is None else np.array(g0, dtype=np.float64)
    ell = 0
    while True:
        lktu = logsumexp(f[:, None] + M, axis=0)
        err = float(np.abs(np.exp(g + lktu) - b).sum())
        if ell >= itr_max or err <= tol:
            break
        g = lb - lktu
        f = la - logsumexp(g[None, :] + M, axis=1)
        ell += 1
    logp = f[:, None] + g[None, :] + M
    w = float((np.exp(logp) * C).sum())
    return SinkhornResult(w, ell, err, f=f, g=g, u=np.exp(f), v=np.exp(g))


def transport_plan(u, v, K) -> np.ndarray:
    """P = diag(u) K diag(v)  (Section 2, Gibbs form of the optimum)."""
    return u[:, None] * K * v[None, :]


def solve_1d(a, b, h: float, eps: float, tol: float, itr_max: int, log: bool = False) -> SinkhornResult:
    n = len(a)
    C = ground_cost_1d(n, h)
    if log:
        return sinkhorn_dense_log(a, b, C, eps, tol, itr_max)
    return sinkhorn_dense(a, b, np.exp(-C / eps), C, tol, itr_max)


def solve_2d(a2, b2, h_fast: float, h_slow: float, eps: float, tol: float, itr_max: int,
             log: bool = False) -> SinkhornResult:
    """a2, b2: (n_slow, n_fast) arrays (fast axis contiguous)."""
    ns, nf = a2.shape
    C = ground_cost_2d(nf, ns, h_fast, h_slow)
    a = np.asarray(a2, dtype=np.float64).reshape(-1)
    b = np.asarray(b2, dtype=np.float64).reshape(-1)
    if log:
        return sinkhorn_dense_log(a, b, C, eps, tol, itr_max)
    return sinkhorn_dense(a, b, np.exp(-C / eps), C, tol, itr_max)


def solve_3d(a3, b3, h, eps: float, tol: float, itr_max: int, log: bool = False) -> SinkhornResult:
    """a3, b3: (n_slow, n_mid, n_fast) arrays (fast axis contiguous);
    h = (h_fast, h_mid, h_slow)."""
    ns, nm, nf = a3.shape
    C = ground_cost_3d(nf, nm, ns, h[0], h[1], h[2])
    a = np.asarray(a3, dtype=np.float64).reshape(-1)
    b = np.asarray(b3, dtype=np.float64).reshape(-1)
    if log:
        return sinkhorn_dense_log(a, b, C, eps, tol, itr_max)
    return sinkhorn_dense(a, b, np.exp(-C / eps), C, tol, itr_max)
