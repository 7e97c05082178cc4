"""Seeded synthetic histograms for the FS-1 workloads.

This module only draws input data. It holds none of the Sinkhorn / FS-1
arithmetic, imports nothing from the rest of the package, and is the one piece
of code shared by the CPU oracle tests and the GPU path.

Every pair is drawn from ``numpy.random.default_rng(SeedSequence([220210042,
workload_id, pair_index]))``; the two histograms a and b of a pair come from
two spawned children of that sequence, so a pair never depends on how many
other pairs were drawn.

Grids are cell centred: x_i = (i + 1/2) h with h = 1/N on [0, 1] (2D: h = 1/side
on both axes).  Densities are evaluated at the cell centres, a floor is added in
density units, and the histogram is normalised to total mass 1 in float64.

Workloads (ids are the ones bench.py takes with --workload):
  1  1D, N = 1000, eps = 1e-2: 2-component Gaussian mixtures,
     mu ~ U[0.2, 0.8], sigma ~ U[0.03, 0.1], floor 1e-4; 1000 iterations.
  2  1D, N = 2^20, eps = 1e-4: 3-component Gaussian mixtures, floor 1e-6;
     tol 1e-6, cap 5000; 256 pairs.
  3  1D uneven batch: N log-uniform in [256, 65536], eps log-uniform in
     [1e-3, 1e-1], Dirichlet(1) weights smoothed by a width-5 box filter
     (zero padded, same size) + floor 1e-6; tol 1e-6, cap 5000; 4096 pairs.
  4  2D, 512 x 512 on [0,1]^2, eps = 1e-3: 1-5 anisotropic Gaussian blobs
     (sigma_x, sigma_y ~ U[0.02, 0.1], theta ~ U[0, pi), centres U[0.2,0.8]^2,
     amplitudes U[0.5, 1]) + floor 1e-7; tol 1e-6, cap 5000; 64 pairs.
  5  serving: Poisson arrivals at 2000 / s for 60 s; half 1D with N
     log-uniform in [1e3, 1e6], half 2D with side log-uniform in [64, 1024];
     smooth Gaussian-mixture histograms; eps log-uniform in [1e-4, 1e-2];
     tol 1e-6, cap 5000.

Replays of the paper's own synthetic experiments (Section 5; their grid is
the node grid x_i = (i - 1) dx - 3, dx = 6 / (N - 1) on [-3, 3] of Section 5.1):
  6  1D random distributions (Section 5.1, Table 1): u_i, v_j ~ U[0, 1],
     normalised to mass 1; eps = 1e-3; 1000 iterations.
  7  Ricker wavelets (Section 5.2, Table 2): R(t) = A (1 - 2 pi^2 f0^2 t^2)
     exp(-pi^2 f0^2 t^2) with f0 = A = 1 and its translate R(t - s),
     s = -1.2032, squared and normalised by eq. "ricker" with delta = 1e-3 and
     L = N (the value that makes the total mass 1); eps = 1e-2; 500
     iterations.  The paper does not state the t-range: the Section 5.1 grid
     is used.
  8  2D random distributions (Section 5.3, Table 3): N x N U[0, 1] values
     normalised to mass 1, h_1 = h_2 = 1, eps = 1e-2; 1000 iterations.

Three axes (the extension stated by the closing remark of Section 4):
  9  3D, 64^3 cells on [0, 1]^3, eps = 2e-3: 1-3 Gaussian blobs + 1e-7;
     tol 1e-6, cap 2000; 32 pairs.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

ROOT_SEED = 220210042


@dataclasses.dataclass
class Problem:
    """One (a, b) pair with its grid and stopping parameters.

    For 2D problems ``a`` and ``b`` have shape (n_slow, n_fast) (row major, the
    fast axis contiguous); ``shape`` is (n_fast, n_slow) and ``h`` is
    (h_fast, h_slow).
    """
    a: np.ndarray
    b: np.ndarray
    h: tuple
    eps: float
    tol: float
    itr_max: int
    ndim: int = 1
    shape: tuple = ()
    workload: int = 0
    index: int = 0
    arrival: float = 0.0

    @property
    def npoints(self) -> int:
        return int(self.a.size)


def _rng_pair(workload: int, index: int):
    ss = np.random.SeedSequence([ROOT_SEED, int(workload), int(index)])
    ca, cb = ss.spawn(2)
    return np.random.default_rng(ca), np.random.default_rng(cb), np.random.default_rng(ss)


def _normalise(rho: np.ndarray) -> np.ndarray:
    rho = np.asarray(rho, dtype=np.float64)
    return rho / rho.sum(dtype=np.float64)


def cell_centres(n: int) -> np.ndarray:
    return (np.arange(n, dtype=np.float64) + 0.5) / n


def gaussian_mixture_1d(rng, n: int, k: int, floor: float,
                        mu_range=(0.2, 0.8), sigma_range=(0.03, 0.1)) -> np.ndarray:
    x = cell_centres(n)
    mu = rng.uniform(*mu_range, size=k)
    sigma = rng.uniform(*sigma_range, size=k)
    rho = np.zeros(n, dtype=np.float64)
    for m, s in zip(mu, sigma):
        rho += np.exp(-0.5 * ((x - m) / s) ** 2) / (s * math.sqrt(2.0 * math.pi))
    rho /= k
    return _normalise(rho + floor)


def dirichlet_box_1d(rng, n: int, width: int, floor: float) -> np.ndarray:
    w = rng.dirichlet(np.ones(n, dtype=np.float64))
    box = np.ones(width, dtype=np.float64) / width
    w = np.convolve(w, box, mode="same")
    return _normalise(n * w + floor)


def blobs_2d(rng, side: int, floor: float, max_blobs: int = 5,
             sigma_range=(0.02, 0.1)) -> np.ndarray:
    """(side, side) image, row major: axis 0 slow (y), axis 1 fast (x)."""
    x = cell_centres(side)
    X = x[None, :]
    Y = x[:, None]
    nb = int(rng.integers(1, max_blobs + 1))
    rho = np.zeros((side, side), dtype=np.float64)
    for _ in range(nb):
        cx, cy = rng.uniform(0.2, 0.8, size=2)
        sx, sy = rng.uniform(*sigma_range, size=2)
        th = rng.uniform(0.0, math.pi)
        amp = rng.uniform(0.5, 1.0)
        c, s = math.cos(th), math.sin(th)
        dx, dy = X - cx, Y - cy
        xr = c * dx + s * dy
        yr = -s * dx + c * dy
        rho += amp * np.exp(-0.5 * ((xr / sx) ** 2 + (yr / sy) ** 2)) / (2.0 * math.pi * sx * sy)
    return _normalise(rho + floor)


# ----------------------------------------------------------------------------
# workloads
# ----------------------------------------------------------------------------

def workload1(index: int = 0, n: int = 1000, eps: float = 1e-2, itr_max: int = 1000) -> Problem:
    ra, rb, _ = _rng_pair(1, index)
    a = gaussian_mixture_1d(ra, n, 2, 1e-4)
    b = gaussian_mixture_1d(rb, n, 2, 1e-4)
    return Problem(a, b, (1.0 / n,), eps, 0.0, itr_max, 1, (n,), 1, index)


def workload2(index: int = 0, n: int = 1 << 20, eps: float = 1e-4, tol: float = 1e-6,
              itr_max: int = 5000) -> Problem:
    ra, rb, _ = _rng_pair(2, index)
    a = gaussian_mixture_1d(ra, n, 3, 1e-6)
    b = gaussian_mixture_1d(rb, n, 3, 1e-6)
    return Problem(a, b, (1.0 / n,), eps, tol, itr_max, 1, (n,), 2, index)


def workload3_params(index: int, n_range=(256, 65536), eps_range=(1e-3, 1e-1)):
    _, _, r = _rng_pair(3, index)
    n = int(round(math.exp(r.uniform(math.log(n_range[0]), math.log(n_range[1])))))
    eps = float(math.exp(r.uniform(math.log(eps_range[0]), math.log(eps_range[1]))))
    return n, eps


def workload3(index: int = 0, tol: float = 1e-6, itr_max: int = 5000,
              n_range=(256, 65536), eps_range=(1e-3, 1e-1)) -> Problem:
    n, eps = workload3_params(index, n_range, eps_range)
    ra, rb, _ = _rng_pair(3, index)
    a = dirichlet_box_1d(ra, n, 5, 1e-6)
    b = dirichlet_box_1d(rb, n, 5, 1e-6)
    return Problem(a, b, (1.0 / n,), eps, tol, itr_max, 1, (n,), 3, index)


def workload4(index: int = 0, side: int = 512, eps: float = 1e-3, tol: float = 1e-6,
              itr_max: int = 5000) -> Problem:
    ra, rb, _ = _rng_pair(4, index)
    a = blobs_2d(ra, side, 1e-7)
    b = blobs_2d(rb, side, 1e-7)
    h = 1.0 / side
    return Problem(a, b, (h, h), eps, tol, itr_max, 2, (side, side), 4, index)


def blobs_3d(rng, side: int, floor: float, max_blobs: int = 3,
             sigma_range=(0.05, 0.15)) -> np.ndarray:
    """(side, side, side) grid, fast axis last: 1-max_blobs axis-aligned
    Gaussian blobs with centres in U[0.2, 0.8]^3, per-axis sigma in
    sigma_range, amplitudes U[0.5, 1], plus a floor, normalised."""
    x = cell_centres(side)
    Z, Y, X = x[:, None, None], x[None, :, None], x[None, None, :]
    nb = int(rng.integers(1, max_blobs + 1))
    rho = np.zeros((side, side, side), dtype=np.float64)
    for _ in range(nb):
        cx, cy, cz = rng.uniform(0.2, 0.8, size=3)
        sx, sy, sz = rng.uniform(*sigma_range, size=3)
        amp = rng.uniform(0.5, 1.0)
        rho += amp * np.exp(-0.5 * (((X - cx) / sx) ** 2 + ((Y - cy) / sy) ** 2 + ((Z - cz) / sz) ** 2))
    return _normalise(rho + floor)


def workload9(index: int = 0, side: int = 64, eps: float = 2e-3, tol: float = 1e-6,
              itr_max: int = 2000) -> Problem:
    """3D grids (the third axis of Section 4's closing remark): side^3 cells on
    [0, 1]^3, 1-3 Gaussian blobs + 1e-7, h = 1/side on every axis."""
    ra, rb, _ = _rng_pair(9, index)
    a = blobs_3d(ra, side, 1e-7)
    b = blobs_3d(rb, side, 1e-7)
    h = 1.0 / side
    return Problem(a, b, (h, h, h), eps, tol, itr_max, 3, (side, side, side), 9, index)


def workload5_arrivals(rate: float = 2000.0, duration: float = 60.0) -> np.ndarray:
    """Poisson arrival times (seconds) of the serving workload."""
    r = np.random.default_rng(np.random.SeedSequence([ROOT_SEED, 5, 0x5E7]))
    t, out = 0.0, []
    while True:
        t += r.exponential(1.0 / rate)
        if t >= duration:
            break
        out.append(t)
    return np.asarray(out, dtype=np.float64)


def workload5(index: int, arrival: float = 0.0, tol: float = 1e-6, itr_max: int = 5000,
              n_range=(1000, 1000000), side_range=(64, 1024),
              eps_range=(1e-4, 1e-2)) -> Problem:
    ra, rb, r = _rng_pair(5, index)
    is2d = bool(r.uniform() < 0.5)
    eps = float(math.exp(r.uniform(math.log(eps_range[0]), math.log(eps_range[1]))))
    if is2d:
        side = int(round(math.exp(r.uniform(math.log(side_range[0]), math.log(side_range[1])))))
        a = blobs_2d(ra, side, 1e-7, max_blobs=3, sigma_range=(0.05, 0.15))
        b = blobs_2d(rb, side, 1e-7, max_blobs=3, sigma_range=(0.05, 0.15))
        h = 1.0 / side
        p = Problem(a, b, (h, h), eps, tol, itr_max, 2, (side, side), 5, index, arrival)
    else:
        n = int(round(math.exp(r.uniform(math.log(n_range[0]), math.log(n_range[1])))))
        a = gaussian_mixture_1d(ra, n, 3, 1e-6)
        b = gaussian_mixture_1d(rb, n, 3, 1e-6)
        p = Problem(a, b, (1.0 / n,), eps, tol, itr_max, 1, (n,), 5, index, arrival)
    return p


def paper_grid(n: int):
    """Node grid of Section 5.1: x_i = (i - 1) dx - 3, dx = 6 / (N - 1)."""
    dx = 6.0 / (n - 1)
    return -3.0 + dx * np.arange(n, dtype=np.float64), dx


def paper_e1(index: int = 0, n: int = 8000, eps: float = 1e-3, itr_max: int = 1000) -> Problem:
    """Section 5.1: U[0, 1] weights on the node grid of [-3, 3], normalised."""
    ra, rb, _ = _rng_pair(6, index)
    a = _normalise(ra.uniform(0.0, 1.0, size=n))
    b = _normalise(rb.uniform(0.0, 1.0, size=n))
    return Problem(a, b, (6.0 / (n - 1),), eps, 0.0, itr_max, 1, (n,), 6, index)


def ricker(t: np.ndarray, f0: float = 1.0, amp: float = 1.0) -> np.ndarray:
    """Ricker wavelet of Section 5.2."""
    q = (math.pi * f0 * t) ** 2
    return amp * (1.0 - 2.0 * q) * np.exp(-q)


def ricker_normalise(f: np.ndarray, delta: float) -> np.ndarray:
    """Eq. "ricker": (f^2 / ||f^2||_1 + delta) / (1 + L delta) with L = N."""
    f2 = f * f
    return (f2 / f2.sum(dtype=np.float64) + delta) / (1.0 + f.size * delta)


def paper_e2(index: int = 0, n: int = 8000, eps: float = 1e-2, itr_max: int = 500,
             shift: float = -1.2032, delta: float = 1e-3) -> Problem:
    """Section 5.2: the Ricker wavelet and its translate (deterministic; the
    index only labels repeats)."""
    x, dx = paper_grid(n)
    a = ricker_normalise(ricker(x), delta)
    b = ricker_normalise(ricker(x - shift), delta)
    return Problem(a, b, (dx,), eps, 0.0, itr_max, 1, (n,), 7, index)


def paper_e3(index: int = 0, side: int = 160, eps: float = 1e-2, itr_max: int = 1000) -> Problem:
    """Section 5.3: N x N U[0, 1] values, h_1 = h_2 = 1, normalised."""
    ra, rb, _ = _rng_pair(8, index)
    a = _normalise(ra.uniform(0.0, 1.0, size=(side, side)))
    b = _normalise(rb.uniform(0.0, 1.0, size=(side, side)))
    return Problem(a, b, (1.0, 1.0), eps, 0.0, itr_max, 2, (side, side), 8, index)


def product_pair_2d(index: int, nx: int, ny: int, floor: float = 1e-3):
    """Separable 2D pair a = a_y (x) a_x, b = b_y (x) b_x, with its 1D factors.

    Used by the 2D product pin: with a separable kernel the 2D iterates factor
    into the 1D ones.  Returns (a2d, b2d, (ax, bx), (ay, by)); 2D arrays are
    (ny, nx) row major.
    """
    ra, rb, _ = _rng_pair(40, index)
    ax = gaussian_mixture_1d(ra, nx, 2, floor)
    ay = gaussian_mixture_1d(ra, ny, 2, floor)
    bx = gaussian_mixture_1d(rb, nx, 2, floor)
    by = gaussian_mixture_1d(rb, ny, 2, floor)
    return np.outer(ay, ax), np.outer(by, bx), (ax, bx), (ay, by)


def product_pair_3d(index: int, nx: int, ny: int, nz: int, floor: float = 1e-3):
    """Separable 3D pair a = a_z (x) a_y (x) a_x (and b likewise) with its 1D
    factors; 3D arrays are (nz, ny, nx), the x axis contiguous."""
    ra, rb, _ = _rng_pair(42, index)
    fa = [gaussian_mixture_1d(ra, n, 2, floor) for n in (nx, ny, nz)]
    fb = [gaussian_mixture_1d(rb, n, 2, floor) for n in (nx, ny, nz)]
    a3 = np.einsum("k,j,i->kji", fa[2], fa[1], fa[0])
    b3 = np.einsum("k,j,i->kji", fb[2], fb[1], fb[0])
    return a3, b3, tuple(zip(fa, fb))


def random_pair_1d(index: int, n: int, floor: float = 0.0, zeros: int = 0):
    """Small generic pair for unit tests: U[0,1] weights (the paper's Section 5.1
    workload shape), optional floor and optional runs of exact zeros."""
    ra, rb, r = _rng_pair(41, index)
    a = ra.uniform(0.0, 1.0, size=n) + floor
    b = rb.uniform(0.0, 1.0, size=n) + floor
    for _ in range(zeros):
        s = int(r.integers(0, max(1, n - 3)))
        ln = int(r.integers(1, max(2, n // 8)))
        a[s:s + ln] = 0.0
        s = int(r.integers(0, max(1, n - 3)))
        b[s:s + ln] = 0.0
    return _normalise(a), _normalise(b)


def batch(workload: int, indices, **kw) -> List[Problem]:
    fn = {1: workload1, 2: workload2, 3: workload3, 4: workload4, 6: paper_e1, 7: paper_e2,
          8: paper_e3, 9: workload9}[workload]
    return [fn(i, **kw) for i in indices]
