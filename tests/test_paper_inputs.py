"""Generators of the paper's own experiments (Section 5): grids and the Ricker
normalisation of eq. "ricker"."""
import math

import numpy as np

from paper_2202_10042_gb300 import inputs


def test_section51_grid():
    x, dx = inputs.paper_grid(7)
    assert dx == 1.0 and x[0] == -3.0 and x[-1] == 3.0
    x, dx = inputs.paper_grid(8000)
    assert abs(x[-1] - 3.0) < 1e-12 and abs(dx - 6.0 / 7999) < 1e-18


def test_ricker_wavelet_values():
    # R(0) = A, zeros at t = +-1 / (sqrt(2) pi f0), minimum -2 A e^{-3/2} at t = +-sqrt(3/2) / (pi f0)
    assert inputs.ricker(np.array([0.0]))[0] == 1.0
    t0 = 1.0 / (math.sqrt(2.0) * math.pi)
    assert abs(inputs.ricker(np.array([t0]))[0]) < 1e-15
    tm = math.sqrt(1.5) / math.pi
    assert abs(inputs.ricker(np.array([tm]))[0] + 2.0 * math.exp(-1.5)) < 1e-15


def test_ricker_normalisation_is_a_probability():
    # eq. "ricker" with L = N: sum (f^2 / ||f^2|| + delta) = 1 + N delta
    p = inputs.paper_e2(0, n=500)
    for h in (p.a, p.b):
        assert abs(h.sum() - 1.0) < 1e-14 and h.min() >= 1e-3 / (1 + 500e-3) - 1e-18
    # R(t - s) is centred at s; the floor's uniform mass (centre 0) dilutes the
    # shift of the mean to s / (1 + N delta)
    x, _ = inputs.paper_grid(500)
    shift = (x * p.b).sum() - (x * p.a).sum()
    assert abs(shift - (-1.2032) / (1 + 500e-3)) < 1e-6


def test_replay_histograms():
    p = inputs.paper_e1(3, n=100)
    assert p.a.shape == (100,) and abs(p.a.sum() - 1) < 1e-14 and p.tol == 0.0 and p.itr_max == 1000
    q = inputs.paper_e3(1, side=12)
    assert q.a.shape == (12, 12) and q.h == (1.0, 1.0) and abs(q.b.sum() - 1) < 1e-14
    assert not np.array_equal(inputs.paper_e1(0, n=50).a, inputs.paper_e1(1, n=50).a)
