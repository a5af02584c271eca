"""Pins of the oracle's synchronous RK3 integrator: on a fixed grid the
solution converges in dt at 3rd order (AB2 at 2nd), the two integrators
approach the same solution, and the low-storage coefficients satisfy the
third-order conditions of an explicit three-stage scheme."""
import math
from fractions import Fraction

import numpy as np

from oracle import ns
from tests import mms


def _run(integrator, dt, T=0.02, N=12):
    fc, _ = mms.exact(1.4, 0.7, 0.05, 0.76)
    cfg = ns.Config(n=(N, N, N), pes=(1, 1, 1), mu0=0.05, dt=dt, integrator=integrator)
    U0 = mms.evaluate(fc, cfg.n, 0.0)
    run = ns.Run.start(cfg, U0, ns.SYNC)
    for _ in range(int(round(T / dt))):
        run.step()
    return run.levels[0]


def _order(integrator):
    dts = (0.004, 0.002, 0.001, 0.0005)
    sols = [_run(integrator, dt) for dt in dts]
    d = [np.max(np.abs(sols[i] - sols[i + 1])) for i in range(3)]
    return [math.log2(d[i] / d[i + 1]) for i in range(2)]


def test_rk3_third_order_in_time():
    o = _order(ns.RK3)
    assert all(2.8 < x < 3.3 for x in o), o


def test_ab2_second_order_in_time():
    o = _order(ns.AB2)
    assert all(1.8 < x < 2.3 for x in o), o


def test_integrators_agree_as_dt_shrinks():
    a = _run(ns.RK3, 0.0005)
    b = _run(ns.AB2, 0.0005)
    assert np.max(np.abs(a - b)) < 1e-6 * np.max(np.abs(a))


def test_low_storage_coefficients_are_third_order():
    """Expand the 2N-storage scheme into its Butcher tableau (exact rationals)
    and check the order conditions sum b = 1, sum b c = 1/2, sum b c^2 = 1/3,
    sum b a c = 1/6."""
    A = [Fraction(0), Fraction(-5, 9), Fraction(-153, 128)]
    B = [Fraction(1, 3), Fraction(15, 16), Fraction(8, 15)]
    # stage increments dU_s = sum_j w[s][j] k_j (k_j = dt R at stage j), U_s = U_0 + sum_j u[s][j] k_j
    w, u = [], [[Fraction(0)] * 3]
    for s in range(3):
        ws = [A[s] * (w[-1][j] if w else 0) + (1 if j == s else 0) for j in range(3)]
        w.append(ws)
        u.append([u[-1][j] + B[s] * ws[j] for j in range(3)])
    a = [u[s] for s in range(3)]        # stage s evaluates R at U_0 + sum_j a[s][j] k_j
    b = u[3]
    c = [sum(a[s]) for s in range(3)]
    assert sum(b) == 1
    assert sum(b[i] * c[i] for i in range(3)) == Fraction(1, 2)
    assert sum(b[i] * c[i] ** 2 for i in range(3)) == Fraction(1, 3)
    assert sum(b[i] * sum(a[i][j] * c[j] for j in range(3)) for i in range(3)) == Fraction(1, 6)
