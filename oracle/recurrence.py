"""FS-1 in pure Python loops: Algorithm 1 and 2 with the Horner / Qin Jiushao
recurrences, the log-domain recurrences and the O(N) transport cost.

Test infrastructure only (see ``oracle/__init__.py``).  Slow on purpose: one
scalar operation per line so that a reader can check it against the paper.
Use it for N up to a few thousand; ``oracle/cref.py`` runs the same
recurrences in C for the large workloads.
"""
from __future__ import annotations

import math

import numpy as np

from .dense import SinkhornResult


# ---------------------------------------------------------------------------
# the matrix-vector product K x as two recurrences
# ---------------------------------------------------------------------------

def horner_matvec(x, lam: float):
    """Section 3, eq. "recursion": K x = p + q with
        p_1 = x_1,  p_{k+1} = lam p_k + x_{k+1}            (lower part, eq. "meshpoly")
        q_N = 0,    q_k = lam (q_{k+1} + x_{k+1})           (strict upper part)
    Returns (p, q)."""
    n = len(x)
    p = [0.0] * n
    q = [0.0] * n
    p[0] = float(x[0])
    for k in range(n - 1):
        p[k + 1] = lam * p[k] + float(x[k + 1])
    q[n - 1] = 0.0
    for k in range(n - 2, -1, -1):
        q[k] = lam * (q[k + 1] + float(x[k + 1]))
    return np.array(p), np.array(q)


def _lse2(x: float, y: float) -> float:
    """log(e^x + e^y), shifted by the larger argument."""
    m = max(x, y)
    if m == -math.inf:
        return -math.inf
    return m + math.log(math.exp(x - m) + math.exp(y - m))


def lse_matvec(f, c: float):
    """Log-domain form of eq. "recursion": with c = h / eps,
        R_1 = f_1,     R_{k+1} = LSE(R_k - c, f_{k+1})
        S_N = -inf,    S_k = LSE(S_{k+1}, f_{k+1}) - c
    so that log(K e^f)_k = LSE(R_k, S_k).  Returns (R, S)."""
    n = len(f)
    R = [0.0] * n
    S = [0.0] * n
    R[0] = float(f[0])
    for k in range(n - 1):
        R[k + 1] = _lse2(R[k] - c, float(f[k + 1]))
    S[n - 1] = -math.inf
    for k in range(n - 2, -1, -1):
        S[k] = _lse2(S[k + 1], float(f[k + 1])) - c
    return np.array(R), np.array(S)


def distance_matvec(x, lam: float):
    """sum_j lam^{|k-j|} |k-j| x_j in O(N) (the return sum of Algorithm 1
    without the factor h).  The paper writes the return as an O(N^2) double
    sum; this is the recurrence form derived for it:
        A_1 = 0,  A_{k+1} = lam (A_k + p_k)           (p from horner_matvec)
        B_N = 0,  B_k = lam (B_{k+1} + q_{k+1} + x_{k+1})
    and the result is A + B."""
    n = len(x)
    p, q = horner_matvec(x, lam)
    A = [0.0] * n
    B = [0.0] * n
    for k in range(n - 1):
        A[k + 1] = lam * (A[k] + p[k])
    for k in range(n - 2, -1, -1):
        B[k] = lam * (B[k + 1] + q[k + 1] + float(x[k + 1]))
    return np.array(A) + np.array(B)


def _lse3(x: float, y: float, z: float) -> float:
    """log(e^x + e^y + e^z), shifted by the largest argument."""
    m = max(x, y, z)
    if m == -math.inf:
        return -math.inf
    return m + math.log(math.exp(x - m) + math.exp(y - m) + math.exp(z - m))


def lse_distance_matvec(g, c: float):
    """Log-domain form of distance_matvec: with x = e^g and lam = e^{-c},
    log(sum_j lam^{|k-j|} |k-j| x_j) for every k (-inf where the sum is 0).
    The four recurrences of horner_matvec / distance_matvec, every quantity
    kept as its logarithm (all of them are sums of non-negative terms):
        P_1 = g_1,       P_{k+1} = LSE(P_k - c, g_{k+1})           (log p)
        A_1 = -inf,      A_{k+1} = LSE(A_k, P_k) - c               (log A)
        Q_N = -inf,      Q_k = LSE(Q_{k+1}, g_{k+1}) - c           (log q)
        B_N = -inf,      B_k = LSE(B_{k+1}, Q_{k+1}, g_{k+1}) - c  (log B)
    and the result is LSE(A_k, B_k).  Unlike distance_matvec it stays finite
    for potentials g of any magnitude."""
    n = len(g)
    P = [0.0] * n
    A = [0.0] * n
    Q = [0.0] * n
    B = [0.0] * n
    P[0] = float(g[0])
    A[0] = -math.inf
    for k in range(n - 1):
        P[k + 1] = _lse2(P[k] - c, float(g[k + 1]))
        A[k + 1] = _lse2(A[k], P[k]) - c
    Q[n - 1] = -math.inf
    B[n - 1] = -math.inf
    for k in range(n - 2, -1, -1):
        Q[k] = _lse2(Q[k + 1], float(g[k + 1])) - c
        B[k] = _lse3(B[k + 1], Q[k + 1], float(g[k + 1])) - c
    return np.logaddexp(np.array(A), np.array(B))


def transport_cost_recurrence(u, v, lam: float, h: float) -> float:
    """sum_ij u_i lam^{|i-j|} |i-j| h v_j via distance_matvec (O(N))."""
    d = distance_matvec(v, lam)
    return float(h * np.dot(np.asarray(u, dtype=np.float64), d))


# ---------------------------------------------------------------------------
# Algorithm 1
# ---------------------------------------------------------------------------

def fs1_plain(a, b, h: float, eps: float, tol: float, itr_max: int) -> SinkhornResult:
    """Algorithm 1 (FS-1), plain form, in the paper's step order:
    lam = e^{-h/eps}; phi = psi = 1/N; while l < itr_max and the column
    marginal error of (phi, psi) exceeds tol: r, s sweeps on phi; psi = v/(r+s);
    p, q sweeps on psi; phi = u/(p+q); l += 1.  Returns the transport cost
    of the final iterate.  (Here a, b are the paper's u, v and u, v are its
    phi, psi.)  The marginal error of the while condition uses K^T phi, which
    is r + s of the same iterate."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    n = a.size
    lam = math.exp(-h / eps)
    u = np.full(n, 1.0 / n)
    v = np.full(n, 1.0 / n)
    ell = 0
    status = 0
    while True:
        r, s = horner_matvec(u, lam)
        ktu = r + s
        err = float(np.abs(v * ktu - b).sum())
        if not math.isfinite(err):
            status = 1
            break
        if ell >= itr_max or err <= tol:
            break
        with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
            v = b / ktu
            p, q = horner_matvec(v, lam)
            u = a / (p + q)
        ell += 1
    w = transport_cost_recurrence(u, v, lam, h) if status == 0 else float("nan")
    return SinkhornResult(w, ell, err, u=u, v=v, status=status)


def fs1_log(a, b, h: float, eps: float, tol: float, itr_max: int) -> SinkhornResult:
    """Algorithm 1 with every iterate absorbed into the potentials (the
    stabilisation of the Remark in Section 3 applied at each step), written
    with the log-domain recurrences of lse_matvec.  f = g = -log N at start."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    n = a.size
    c = h / eps
    with np.errstate(divide="ignore"):
        la = np.log(a)
        lb = np.log(b)
    f = np.full(n, -math.log(n))
    g = np.full(n, -math.log(n))
    ell = 0
    while True:
        R, S = lse_matvec(f, c)
        lktu = np.logaddexp(R, S)
        err = float(np.abs(np.exp(g + lktu) - b).sum())
        if ell >= itr_max or err <= tol:
            break
        g = lb - lktu
        P, Q = lse_matvec(g, c)
        f = la - np.logaddexp(P, Q)
        ell += 1
    lam = math.exp(-c)
    # transport cost with the potentials shifted to keep exp() in range
    mf, mg = np.max(f), np.max(g)
    w = transport_cost_recurrence(np.exp(f - mf), np.exp(g - mg), lam, h) * math.exp(mf + mg)
    return SinkhornResult(w, ell, err, f=f, g=g, u=np.exp(f), v=np.exp(g))


def fs1_stabilised(a, b, h: float, eps: float, tol: float, itr_max: int,
                   tau: float = 1e10) -> SinkhornResult:
    """Algorithm 1 with the log-domain stabilisation of the Remarks in
    Sections 2 and 3.  State: absorbed potentials A = alpha/eps, B = beta/eps
    and residual scalings phi~, psi~ (true u = e^A phi~, v = e^B psi~).  When
    ||phi~||_inf or ||psi~||_inf exceeds tau, A += log phi~, B += log psi~ and
    phi~ = psi~ = 1.  The sweeps use the rescaled recurrences of the Remark in
    Section 3 (its replaced lines 5, 6, 10, 11):
        r_{i+1} = lam e^{B_{i+1}-B_i} r_i + e^{A_{i+1}+B_{i+1}} phi~_{i+1}
        s_{i}   = lam e^{B_i-B_{i+1}} (s_{i+1} + e^{A_{i+1}+B_{i+1}} phi~_{i+1})
    and the same with A, B swapped for p, q.  The first terms r_1, p_1 carry
    the factor e^{A_1+B_1} as well (the Remark leaves lines 3 and 9 as
    written; with the rescaled kernel they must carry it).  Requires a, b > 0.
    """
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    n = a.size
    lam = math.exp(-h / eps)
    A = np.zeros(n)
    B = np.zeros(n)
    ph = np.full(n, 1.0 / n)
    ps = np.full(n, 1.0 / n)

    def sweep(x, S):
        # y_i = e^{S_i} sum_j lam^{|i-j|} e^{-S_j} x_j with the rescaled recurrences
        r = [0.0] * n
        s = [0.0] * n
        r[0] = x[0]
        for i in range(n - 1):
            r[i + 1] = lam * math.exp(S[i + 1] - S[i]) * r[i] + x[i + 1]
        s[n - 1] = 0.0
        for i in range(n - 2, -1, -1):
            s[i] = lam * math.exp(S[i] - S[i + 1]) * (s[i + 1] + x[i + 1])
        return np.array(r) + np.array(s)

    ell = 0
    while True:
        if max(np.max(np.abs(ph)), np.max(np.abs(ps))) > tau:
            A = A + np.log(ph)
            B = B + np.log(ps)
            ph = np.ones(n)
            ps = np.ones(n)
        eab = np.exp(A + B)
        ktu = sweep(eab * ph, B)            # = e^B * K^T (e^A phi~)
        err = float(np.abs(ps * ktu - b).sum())
        if ell >= itr_max or err <= tol:
            break
        ps = b / ktu
        kv = sweep(eab * ps, A)             # = e^A * K (e^B psi~)
        ph = a / kv
        ell += 1
    f = A + np.log(ph)
    g = B + np.log(ps)
    mf, mg = np.max(f), np.max(g)
    w = transport_cost_recurrence(np.exp(f - mf), np.exp(g - mg), lam, h) * math.exp(mf + mg)
    return SinkhornResult(w, ell, err, f=f, g=g)


# ---------------------------------------------------------------------------
# Algorithm 2 (2D)
# ---------------------------------------------------------------------------

def horner_matvec_2d(x2, lam1: float, lam2: float):
    """Section 4, eq. "2d recursion": K x for K = [lam2^{|k-l|} K_0] on an
    (n_slow, n_fast) array (row l = the paper's column vector psi_l of length
    N).  Each row is multiplied by K_0 with the 1D recurrences, then the
    block recurrences with lam2 run across rows:
        p_1 = K_0 x_1,   p_{k+1} = lam2 p_k + K_0 x_{k+1}
        q_M = 0,         q_k = lam2 (q_{k+1} + K_0 x_{k+1})."""
    x2 = np.asarray(x2, dtype=np.float64)
    M, N = x2.shape
    k0x = []
    for l in range(M):
        p, q = horner_matvec(x2[l], lam1)
        k0x.append(p + q)
    P = [None] * M
    Q = [None] * M
    P[0] = k0x[0]
    for k in range(M - 1):
        P[k + 1] = lam2 * P[k] + k0x[k + 1]
    Q[M - 1] = np.zeros(N)
    for k in range(M - 2, -1, -1):
        Q[k] = lam2 * (Q[k + 1] + k0x[k + 1])
    return np.array(P) + np.array(Q)


def fs1_plain_2d(a2, b2, h_fast: float, h_slow: float, eps: float, tol: float,
                 itr_max: int) -> SinkhornResult:
    """Algorithm 2 (2D FS-1), plain form.  a2, b2 are (n_slow, n_fast)."""
    a2 = np.asarray(a2, dtype=np.float64)
    b2 = np.asarray(b2, dtype=np.float64)
    M, N = a2.shape
    lam1 = math.exp(-h_fast / eps)
    lam2 = math.exp(-h_slow / eps)
    u = np.full((M, N), 1.0 / (N * M))
    v = np.full((M, N), 1.0 / (N * M))
    ell = 0
    while True:
        ktu = horner_matvec_2d(u, lam1, lam2)
        err = float(np.abs(v * ktu - b2).sum())
        if ell >= itr_max or err <= tol:
            break
        v = b2 / ktu
        u = a2 / horner_matvec_2d(v, lam1, lam2)
        ell += 1
    # return sum of Algorithm 2, split by the two terms of the cost:
    # h1 |i1-i2| weighted along the fast axis then the plain slow kernel, and
    # the plain fast kernel then h2 |j1-j2| weighted along the slow axis.
    d_fast = np.array([distance_matvec(v[l], lam1) for l in range(M)])
    t1 = _slow_apply(d_fast, lam2, weighted=False)
    k0v = np.array([sum(horner_matvec(v[l], lam1)) for l in range(M)])
    t2 = _slow_apply(k0v, lam2, weighted=True)
    w = float((u * (h_fast * t1 + h_slow * t2)).sum())
    return SinkhornResult(w, ell, err, u=u, v=v)


def _slow_apply(rows, lam2: float, weighted: bool):
    """Apply lam2^{|k-l|} (times |k-l| when weighted) across the slow axis."""
    rows = np.asarray(rows, dtype=np.float64)
    M, N = rows.shape
    out = np.zeros((M, N))
    for col in range(N):
        x = rows[:, col]
        if weighted:
            out[:, col] = distance_matvec(x, lam2)
        else:
            p, q = horner_matvec(x, lam2)
            out[:, col] = p + q
    return out
