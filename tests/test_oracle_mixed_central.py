"""Pins of the other reading of the mixed derivatives at PE faces
(Config.mixed_central): the central a-stencil of d/dx_a (d u/dx_b) at every
point, where the stencil points beyond an a-face of delay k take the
neighbour's b-derivative extrapolated to level n with the Table B weights
(sum_l w_l(k) D_b u^{n-k-l}, D_b the plain central stencil of the whole level;
under extrapolate_state, D_b of u of the extrapolated state) instead of the
three-step rule's one-sided stencils (Sec. 2.1).

* Without delays it is the single-PE scheme bit for bit (4th and 6th order,
  either extrapolation reading), where the three-step rule is not.
* Under random delays it converges at the scheme's order on the manufactured
  solution whose mixed viscous terms are nonzero (tests/mms.py, mixed=True;
  4th order, 6th for the 6th-order scheme); with the neighbour's gradient
  taken from level n-k without extrapolation it does not (a planted mistake:
  the momentum orders fall to about 1).
* It equals its pointwise brute force (oracle/pointwise.py), which builds
  each term per point.
"""
import math

import numpy as np
import pytest

from oracle import ns
from oracle.pointwise import PointOracle
from paper_2003_10561_gb300 import synth
from tests import mms

GAMMA, PR, MU0, OMEGA = 1.4, 0.7, 0.05, 0.76


def _cfg(N, pes, **kw):
    base = dict(n=(N, N, N), pes=pes, gamma=GAMMA, prandtl=PR, mu0=MU0, visc_exp=OMEGA, max_delay=2,
                mixed_central=True)
    base.update(kw)
    return ns.Config(**base)


@pytest.mark.parametrize("order,xstate", [(4, False), (4, True), (6, False)])
def test_zero_delay_is_the_single_pe_scheme(order, xstate):
    N = 16 if order == 4 else 21
    U = synth.initial_state((N, N, N), k0=3.0, mach_t=0.3, seed=2)
    one = _cfg(N, (1, 1, 1), order=order, mixed_central=False)
    R1 = ns.rhs(one, [U] * one.n_levels, np.zeros((1, 6), dtype=int))
    pes = (2, 2, 2) if order == 4 else (3, 1, 3)
    c = _cfg(N, pes, order=order, extrapolate_state=xstate)
    hist = synth.history(U, c.n_levels, eps=2e-2, seed=3)
    hist[0] = U                      # older levels differ; zero delays read level n only
    zero = np.zeros((c.n_pes, 6), dtype=int)
    assert np.array_equal(ns.rhs(c, hist, zero), R1)
    # the three-step rule's one-sided stencils differ from the single-PE scheme
    d = ns.rhs(_cfg(N, pes, order=order, mixed_central=False), hist, zero)
    assert np.max(np.abs(d[1] - R1[1])) > 1e-6 * np.max(np.abs(R1[1]))


def _mms_orders(order, Ns, **kw):
    fc, fr = mms.exact(GAMMA, PR, MU0, OMEGA, mixed=True)
    errs = []
    for N in Ns:
        cfg = _cfg(N, (2, 2, 2), order=order, **kw)
        dt = 0.5 * (2 * math.pi / N) ** 2
        levels = [mms.evaluate(fc, cfg.n, 0.4 - l * dt) for l in range(cfg.n_levels)]
        delays = ns.delay_map(ns.Config(**{**cfg.__dict__, "seed": 17}), 50, ns.RANDOM)
        R = ns.rhs(cfg, levels, delays)
        Rex = mms.evaluate(fr, cfg.n, 0.4)
        errs.append([float(np.max(np.abs(R[v] - Rex[v])) / np.max(np.abs(Rex[v]))) for v in range(5)])
    orders = [math.log(errs[-2][v] / errs[-1][v]) / math.log(Ns[-1] / Ns[-2]) for v in range(5)]
    return orders, errs


@pytest.mark.parametrize("xstate", [False, True])
def test_manufactured_solution_fourth_order_under_delays(xstate):
    orders, errs = _mms_orders(4, (16, 32, 64), extrapolate_state=xstate)
    assert min(orders) > 3.5, (orders, errs)


def test_manufactured_solution_sixth_order_under_delays():
    orders, errs = _mms_orders(6, (16, 32, 48))
    assert min(orders) > 5.3, (orders, errs)


def test_unextrapolated_neighbour_gradient_is_detected(monkeypatch):
    """The neighbour's gradient of level n-k taken as it is (no Table B
    weights) is O(k dt) = O(dx^2) off; the central a-stencil divides that by
    dx, and the order falls well below 4."""
    sc4 = ns.Config(n=(8, 8, 8)).scheme

    def stale(cfg, flevels, b):
        den = sc4.d1_den * cfg.dx[b]
        return [ns._apply(flevels[k], sc4.d1, ns._axis(b)) / den for k in range(cfg.max_delay + 1)]

    monkeypatch.setattr(ns, "ghost_gradients", stale)
    orders, errs = _mms_orders(4, (16, 32, 64))
    assert min(orders) < 3.0, (orders, errs)


def test_readings_differ_under_delays():
    N = 16
    U = synth.initial_state((N, N, N), k0=3.0, mach_t=0.3, seed=5)
    c = _cfg(N, (2, 2, 2), seed=9)
    hist = synth.history(U, c.n_levels, eps=2e-2, seed=6)
    d = ns.delay_map(c, 20, ns.RANDOM)
    a = ns.rhs(c, hist, d)
    b = ns.rhs(_cfg(N, (2, 2, 2), seed=9, mixed_central=False), hist, d)
    assert np.array_equal(a[0], b[0])                 # continuity has no viscous term
    assert np.max(np.abs(a[1] - b[1])) > 1e-6 * np.max(np.abs(a[1]))


@pytest.mark.parametrize("N,pes,order,xstate", [(12, (2, 2, 2), 4, False), (12, (3, 1, 2), 4, True),
                                                (14, (2, 1, 2), 6, False)])
def test_brute_force_pointwise_matches_vectorised(N, pes, order, xstate):
    cfg = _cfg(N, pes, order=order, extrapolate_state=xstate, seed=5, forcing=True, kf=2.0, f_amp=0.05,
               f_tcorr=0.5, dt=0.01, f_seed=9)
    U = synth.initial_state(cfg.n, k0=3.0, mach_t=0.3, seed=4)
    hist = synth.history(U, cfg.n_levels, eps=2e-2)
    delays = ns.delay_map(cfg, 30, ns.RANDOM)
    fh = ns.forcing_coefficients(cfg, 3)
    R = ns.rhs(cfg, hist, delays, fh)
    po = PointOracle(cfg, lambda l: hist[l], delays, fh, ns.forcing_modes(cfg.kf))
    rng = np.random.default_rng(0)
    pts = [tuple(int(v) for v in rng.integers(0, N, 3)) for _ in range(30)]
    pts += [(0, 0, 0), (N - 1, N - 1, N - 1), (1, 5, 6), (5, 6, 1)]
    scale = np.abs(R).max(axis=(1, 2, 3))
    for (x, y, z) in pts:
        r = po.rhs((x, y, z))
        for v in range(5):
            assert abs(r[v] - R[v, z, y, x]) <= 1e-13 * scale[v], (x, y, z, v)
