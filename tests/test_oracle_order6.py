"""Pins of the oracle's 6th-order AT scheme (Table B rows (1,6) and (2,6)).

* The central and one-sided 6th-order stencils are exact on polynomials of
  degree <= 6 (the central D2 up to 7) and not beyond: exact integer sums of
  c_o o^m.
* The T_l = 4 weights are the cubic Lagrange extrapolation from the levels
  n-k .. n-k-3 to level n, derived here with exact rationals; they are
  (1, 0, 0, 0) at k = 0.
* The AT derivative keeps 6th order at PE faces under delays with dt ~ dx^2,
  where a 4th-order AT scheme stays at 4th order.
* The full right-hand side converges at 6th order to the sympy exact RHS with
  one PE, with 2x2x2 PEs synchronously (one-sided 6th-order mixed derivatives)
  and with 2x2x2 PEs under random delays.
* The brute-force pointwise evaluation equals the vectorised one.
* Start-up: delays stay zero for the first L + 4 steps.
"""
from fractions import Fraction
import math

import numpy as np
import pytest

from oracle import ns
from oracle.pointwise import PointOracle
from oracle.stencils import Scheme, at_weights6
from paper_2003_10561_gb300 import synth
from tests import mms

SC = Scheme(6)
GAMMA, PR, MU0, OMEGA = 1.4, 0.7, 0.05, 0.76


def _moment(stencil, m):
    return sum(Fraction(int(c)) * Fraction(o) ** m for o, c in stencil)


@pytest.mark.parametrize("li", [0, 1, 2, 9, 10, 11, 5])
def test_first_derivative_stencils_exact_to_degree_six(li):
    st = SC.one_sided(li, 12)
    assert len(st) in (6, 7)
    for m in range(7):
        # sum c o^m = den * d/dx (x^m) at 0 = den * [m == 1]
        assert _moment(st, m) == (Fraction(60) if m == 1 else 0), (li, m)
    assert _moment(st, 7) != 0
    # a PE-local stencil never reaches outside the PE
    assert all(0 <= li + o < 12 for o, _ in st)


def test_second_derivative_stencil_exact_to_degree_seven():
    for m in range(8):
        assert _moment(SC.d2, m) == (Fraction(360) if m == 2 else 0), m
    assert _moment(SC.d2, 8) != 0


def _lagrange_at_zero(k, T):
    nodes = [Fraction(-(k + l)) for l in range(T)]
    w = []
    for l in range(T):
        num = den = Fraction(1)
        for m in range(T):
            if m != l:
                num *= -nodes[m]
                den *= nodes[l] - nodes[m]
        w.append(num / den)
    return w


@pytest.mark.parametrize("k", range(7))
def test_weights_are_cubic_lagrange_extrapolation(k):
    w = at_weights6(k)
    lag = _lagrange_at_zero(k, 4)
    assert [Fraction(v) for v in w] == lag
    assert sum(w) == 1.0
    if k == 0:
        assert w == (1.0, 0.0, 0.0, 0.0)
    # exact for cubics in time, not for quartics (k > 0)
    for m in range(4):
        assert sum(Fraction(w[l]) * Fraction(-(k + l)) ** m for l in range(4)) == (1 if m == 0 else 0)
    if k > 0:
        assert sum(Fraction(w[l]) * Fraction(-(k + l)) ** 4 for l in range(4)) != 0


def _wave_levels(N, n_levels, cfl_d=0.5, kx=1):
    h = 2 * math.pi / N
    dt = cfl_d * h * h
    x = np.arange(N) * h
    tn = 0.3
    lev = [np.broadcast_to(np.sin(kx * (x - (tn - l * dt))), (4, 4, N)).copy() for l in range(n_levels)]
    return lev, kx * np.cos(kx * (x - tn)), -kx * kx * np.sin(kx * (x - tn))


@pytest.mark.parametrize("deriv", [1, 2])
def test_at_sixth_order_under_delay(deriv):
    """Delays k = L on every face, dt = 0.5 dx^2: the error at the PE-face
    points falls at 6th order (the 4th-order scheme at 4th)."""
    L = 2
    for order, expect in ((6, 5.5), (4, 3.6)):
        errs = []
        for N in (32, 64, 128):
            cfg = ns.Config(n=(N, 4, 4), pes=(4, 1, 1), max_delay=L, order=order)
            lev, e1, e2 = _wave_levels(N, cfg.n_levels)
            d = ns.at_derivative(cfg, lev, 0, np.full((cfg.n_pes, 6), L), deriv)[0, 0]
            li = np.arange(N) % cfg.nloc[0]
            M = cfg.scheme.M
            face = (li < M) | (li >= cfg.nloc[0] - M)
            errs.append(np.max(np.abs(d - (e1 if deriv == 1 else e2))[face]))
        orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
        assert all(o > expect for o in orders), (order, errs, orders)
        if order == 4:
            assert all(o < 4.6 for o in orders), orders


def test_start_up_is_synchronous_for_l_plus_four_steps():
    cfg = ns.Config(n=(16, 16, 16), pes=(2, 2, 2), max_delay=3, seed=4, order=6)
    assert cfg.n_levels == 7
    for n in range(7):
        assert not ns.delay_map(cfg, n, ns.RANDOM).any()
        assert not ns.delay_map(cfg, n, ns.PERIODIC).any()
    assert ns.delay_map(cfg, 7, ns.RANDOM).any()
    assert (ns.delay_map(cfg, 8, ns.PERIODIC) == 1).all()


def _mms_error(N, pes, random, mixed=False):
    fc, fr = mms.exact(GAMMA, PR, MU0, OMEGA, mixed=mixed)
    cfg = ns.Config(n=(N, N, N), pes=pes, gamma=GAMMA, prandtl=PR, mu0=MU0, visc_exp=OMEGA,
                    max_delay=2, order=6, seed=17)
    dt = 0.5 * (2 * math.pi / N) ** 2
    levels = [mms.evaluate(fc, cfg.n, 0.4 - l * dt) for l in range(cfg.n_levels)]
    delays = ns.delay_map(cfg, 50, ns.RANDOM) if random else np.zeros((cfg.n_pes, 6), dtype=int)
    R = ns.rhs(cfg, levels, delays)
    Rex = mms.evaluate(fr, cfg.n, 0.4)
    return [float(np.max(np.abs(R[v] - Rex[v])) / np.max(np.abs(Rex[v]))) for v in range(5)]


@pytest.mark.parametrize("pes,random", [((1, 1, 1), False), ((2, 2, 2), False), ((2, 2, 2), True)],
                         ids=["one-PE", "2x2x2-sync", "2x2x2-random"])
def test_manufactured_solution_sixth_order(pes, random):
    errs = [_mms_error(N, pes, random) for N in (16, 32, 48)]
    for v in range(5):
        o = math.log(errs[1][v] / errs[2][v]) / math.log(48 / 32)
        assert o > 5.3, (v, errs, o)
    assert max(errs[2]) < 2e-6


def test_manufactured_solution_sixth_order_with_mixed_terms():
    """The field set whose mixed viscous terms are nonzero (in the other one
    they vanish): the three-step rule with the 7-point one-sided rows keeps
    6th order under random delays (measured 5.91-5.97)."""
    errs = [_mms_error(N, (2, 2, 2), True, mixed=True) for N in (32, 48)]
    for v in range(5):
        o = math.log(errs[0][v] / errs[1][v]) / math.log(48 / 32)
        assert o > 5.3, (v, errs, o)


@pytest.mark.parametrize("pes", [(2, 2, 2), (3, 1, 2)])
def test_brute_force_pointwise_matches_vectorised(pes):
    N = 14 if pes[0] == 2 else 21
    n = (N, 14, 14)
    cfg = ns.Config(n=n, pes=pes, gamma=GAMMA, prandtl=PR, mu0=MU0, visc_exp=OMEGA, max_delay=3, order=6,
                    forcing=True, kf=2.0, f_amp=0.05, f_tcorr=0.5, dt=0.01, f_seed=9, seed=5)
    U = synth.initial_state(n, k0=3.0, mach_t=0.3, seed=4, gamma=GAMMA)
    hist = synth.history(U, cfg.n_levels, eps=2e-2)
    delays = ns.delay_map(cfg, 30, ns.RANDOM)
    assert delays.max() == 3
    fh = ns.forcing_coefficients(cfg, 3)
    R = ns.rhs(cfg, hist, delays, fh)
    po = PointOracle(cfg, lambda l: hist[l], delays, fh, ns.forcing_modes(cfg.kf))
    rng = np.random.default_rng(0)
    pts = [tuple(int(rng.integers(0, n[d])) for d in range(3)) for _ in range(50)]
    pts += [(0, 0, 0), (n[0] - 1, 13, 13), (2, 6, 7), (7, 3, 4), (6, 0, 11)]
    scale = np.abs(R).max(axis=(1, 2, 3))
    for (x, y, z) in pts:
        r = po.rhs((x, y, z))
        for v in range(5):
            assert abs(r[v] - R[v, z, y, x]) <= 1e-13 * scale[v], (x, y, z, v)


def test_boundary_fraction_uses_three_layers():
    cfg = ns.Config(n=(64, 64, 64), pes=(4, 4, 4), order=6)
    assert abs(ns.boundary_fraction(cfg) - (1 - (10 / 16) ** 3)) < 1e-15
