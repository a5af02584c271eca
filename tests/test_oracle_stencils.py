"""Pins of the oracle's stencils and AT weights against closed forms.

* central D1 / D2 and the one-sided D1 stencils are exact on polynomials of
  degree <= 4 (4th order);
* on sin(m x) the periodic central stencils give the closed-form modified
  wavenumbers (checks offsets and signs of the roll);
* the Table B weights sum to one, are (1, 0, 0) at k = 0 and extrapolate
  quadratics in time exactly (and no cubic), i.e. they are the quadratic
  Lagrange extrapolation from levels n-k, n-k-1, n-k-2;
* the AT derivative keeps 4th order under delay with dt ~ dx^2
  (Sec. 2.1, Eq. (at22) remark), while the standard stencil with a delayed
  neighbour collapses to zeroth order for the second derivative
  (Sec. 2, Eq. (d2as));
* conservation: the sum over a periodic line of AT first derivatives of a
  smooth f(x, t) is O(dx^5) under delays (Eq. (ts4)) and zero to round-off
  without them.
"""
import math

import numpy as np
import pytest

from oracle import ns
from oracle.stencils import (D1_CENTRAL, D2_CENTRAL, D1_FORWARD0, D1_FORWARD1,
                             D1_BACKWARD0, D1_BACKWARD1, at_weights,
                             d1_central_periodic, d2_central_periodic)


def _apply_at(stencil, f, x0, h):
    return sum(c * f(x0 + o * h) for o, c in stencil)


@pytest.mark.parametrize("deg", range(5))
def test_polynomial_exactness(deg):
    rng = np.random.default_rng(deg)
    a = rng.standard_normal(deg + 1)
    f = np.polynomial.Polynomial(a)
    df, d2f = f.deriv(1), f.deriv(2)
    h, x0 = 0.37, 0.81
    for st in (D1_CENTRAL, D1_FORWARD0, D1_FORWARD1, D1_BACKWARD0, D1_BACKWARD1):
        assert abs(_apply_at(st, f, x0, h) / (12 * h) - df(x0)) < 1e-11
    assert abs(_apply_at(D2_CENTRAL, f, x0, h) / (12 * h * h) - d2f(x0)) < 1e-10


def test_degree5_not_exact():
    f = np.polynomial.Polynomial([0, 0, 0, 0, 0, 1.0])
    h = 0.3
    assert abs(_apply_at(D1_CENTRAL, f, 0.5, h) / (12 * h) - f.deriv(1)(0.5)) > 1e-6
    assert abs(_apply_at(D1_FORWARD0, f, 0.5, h) / (12 * h) - f.deriv(1)(0.5)) > 1e-6


@pytest.mark.parametrize("m", [1, 3, 7])
def test_modified_wavenumber(m):
    N = 32
    h = 2 * math.pi / N
    x = np.arange(N) * h
    f = np.broadcast_to(np.sin(m * x), (2, 3, N)).copy()
    d1 = d1_central_periodic(f, 2, h)[0, 0]
    d2 = d2_central_periodic(f, 2, h)[0, 0]
    k1 = (8 * math.sin(m * h) - math.sin(2 * m * h)) / (6 * h)
    k2 = (32 * math.cos(m * h) - 2 * math.cos(2 * m * h) - 30) / (12 * h * h)
    assert np.allclose(d1, k1 * np.cos(m * x), atol=1e-12)
    assert np.allclose(d2, k2 * np.sin(m * x), atol=1e-11)


def test_central_convergence_order_four():
    errs = []
    for N in (32, 64, 128):
        h = 2 * math.pi / N
        x = np.arange(N) * h
        f = np.broadcast_to(np.exp(np.sin(x)), (1, 1, N)).copy()
        d1 = d1_central_periodic(f, 2, h)[0, 0]
        errs.append(np.max(np.abs(d1 - np.cos(x) * np.exp(np.sin(x)))))
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(3.85 < o < 4.2 for o in orders), orders


def test_at_weights_table_b():
    assert at_weights(0) == (1.0, 0.0, 0.0)
    assert at_weights(1) == (3.0, -3.0, 1.0)
    assert at_weights(2) == (6.0, -8.0, 3.0)
    for k in range(6):
        assert sum(at_weights(k)) == 1.0


@pytest.mark.parametrize("k", range(5))
def test_at_weights_quadratic_extrapolation(k):
    w = at_weights(k)
    rng = np.random.default_rng(k)
    for _ in range(3):
        a, b, c = rng.standard_normal(3)
        g = lambda s: a + b * s + c * s * s     # s = time level offset from n
        ext = sum(w[l] * g(-(k + l)) for l in range(3))
        assert abs(ext - g(0)) < 1e-12 * (1 + abs(g(-k)) * (k + 3) ** 2)
    if k > 0:
        cub = lambda s: s ** 3
        assert abs(sum(w[l] * cub(-(k + l)) for l in range(3)) - cub(0)) > 0.5


def _wave_levels(N, cfl_d, n_levels, c=1.0, kx=1):
    """q(x, t) = sin(kx (x - c t)) at levels t_n - l dt, dt = cfl_d dx^2."""
    h = 2 * math.pi / N
    dt = cfl_d * h * h
    x = np.arange(N) * h
    tn = 0.3
    lev = []
    for l in range(n_levels):
        t = tn - l * dt
        lev.append(np.broadcast_to(np.sin(kx * (x - c * t)), (4, 4, N)).copy())
    exact_d1 = kx * np.cos(kx * (x - c * tn))
    exact_d2 = -kx * kx * np.sin(kx * (x - c * tn))
    return lev, exact_d1, exact_d2


def _line_cfg(N, P, L):
    return ns.Config(n=(N, 4, 4), pes=(P, 1, 1), max_delay=L)


@pytest.mark.parametrize("order", [1, 2])
def test_at_order_of_accuracy_under_delay(order):
    """Delays k = L on every face, dt = 0.5 dx^2: the AT derivative error at the
    PE-face points falls at 4th order (Sec. 2.1)."""
    L = 2
    errs = []
    for N in (32, 64, 128):
        cfg = _line_cfg(N, 4, L)
        lev, e1, e2 = _wave_levels(N, 0.5, cfg.n_levels)
        delays = np.full((cfg.n_pes, 6), L)
        d = ns.at_derivative(cfg, lev, 0, delays, order)[0, 0]
        exact = e1 if order == 1 else e2
        li = np.arange(N) % cfg.nloc[0]
        face = (li < 2) | (li >= cfg.nloc[0] - 2)
        errs.append(np.max(np.abs(d - exact)[face]))
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(o > 3.6 for o in orders), (errs, orders)


def test_delayed_standard_stencil_is_zeroth_order():
    """The standard D2 with the neighbour across the face at level n-k
    (Eq. (d2as)) does not converge: its error stays O(1) as dx -> 0."""
    errs = []
    for N in (32, 64, 128):
        h = 2 * math.pi / N
        lev, _, e2 = _wave_levels(N, 0.5, 3)
        # point i = first of a PE; left neighbours at level n-1, right at n
        i = N // 2
        f0, f1 = lev[0][0, 0], lev[1][0, 0]
        d2 = (-f1[i - 2] + 16 * f1[i - 1] - 30 * f0[i] + 16 * f0[i + 1] - f0[i + 2]) / (12 * h * h)
        errs.append(abs(d2 - e2[i]))
    assert errs[-1] > 0.3 * errs[0]          # no decay with resolution
    assert errs[-1] > 1e-2


def test_zero_delay_reduces_exactly():
    """k = 0 on every face: the AT derivative equals the standard periodic
    stencil bit for bit (Sec. 2.1)."""
    N = 48
    cfg = _line_cfg(N, 4, 2)
    rng = np.random.default_rng(5)
    lev = [rng.standard_normal((4, 4, N)) for _ in range(cfg.n_levels)]
    delays = np.zeros((cfg.n_pes, 6), dtype=int)
    h = cfg.dx[0]
    a = ns.at_derivative(cfg, lev, 0, delays, 1)
    b = ns.at_derivative(ns.Config(n=(N, 4, 4), pes=(1, 1, 1)), lev, 0, delays[:1], 1)
    assert np.array_equal(a, b)
    assert np.allclose(b, d1_central_periodic(lev[0], 2, h), rtol=0, atol=1e-12)


def test_conservation_residual_order_five():
    """sum_i D1^AT f_i over a periodic line is O(dx^5) with delays and dt ~ dx^2
    (Eq. (ts4)), and zero to round-off without delays."""
    res = []
    for N in (64, 128, 256):
        cfg = _line_cfg(N, 4, 2)
        lev, _, _ = _wave_levels(N, 0.5, cfg.n_levels, kx=2)
        delays = np.zeros((cfg.n_pes, 6), dtype=int)
        d0 = ns.at_derivative(cfg, lev, 0, delays, 1)[0, 0]
        assert abs(d0.sum()) < 1e-11
        delays[:, 0] = [1, 2, 0, 2]
        delays[:, 1] = [2, 1, 1, 0]
        d = ns.at_derivative(cfg, lev, 0, delays, 1)[0, 0]
        res.append(abs(d.sum()))
    orders = [math.log2(res[i] / res[i + 1]) for i in range(2)]
    assert all(o > 4.6 for o in orders), (res, orders)
