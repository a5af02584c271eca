"""Pins of the oracle's right-hand side.

* Manufactured solution: on smooth fields the oracle RHS converges at 4th order
  to the exact RHS that sympy derives from the PDEs in divergence form -- with
  one PE, with 2x2x2 PEs synchronously, and with 2x2x2 PEs under random delays
  whose past levels are the exact solution at t - l dt, dt ~ dx^2 (Sec. 2.1).
  A dropped term, a wrong sign or a transposed index breaks the convergence.
* Conservation (Sec. 2.1): sum R_rho = 0 to round-off in every mode without
  delays; all five sums vanish to round-off in the Euler limit (mu = 0).
* Exact reduction at k = 0: with synchronous delays and mu = 0 the 2x2x2-PE RHS
  equals the single-PE RHS bit for bit.
* Kinetic-energy budget (Eq. (meantke)): dK/dt from the RHS matches
  <p theta> - <sigma_ij S_ij> + <rho f_i u_i> at 4th order.
* Brute force: the vectorised RHS equals the pointwise Table B term sums.
* The other reading of the extrapolation (the state extrapolated first, the
  quantity evaluated once): equal to the default without delays and for the
  linear continuity fluxes, exact on a steady history, 4th order on the
  manufactured solution under random delays, and equal to its own pointwise
  brute force.
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
    base = dict(n=(N, N, N), pes=pes, gamma=GAMMA, prandtl=PR, mu0=MU0, visc_exp=OMEGA, max_delay=2)
    base.update(kw)
    return ns.Config(**base)


def _mms_error(N, pes, delays_fn=None, cdt=0.5):
    fc, fr = mms.exact(GAMMA, PR, MU0, OMEGA)
    cfg = _cfg(N, pes)
    dx = 2 * math.pi / N
    dt = cdt * dx * dx
    tn = 0.4
    levels = [mms.evaluate(fc, cfg.n, tn - l * dt) for l in range(cfg.n_levels)]
    delays = delays_fn(cfg) if delays_fn else np.zeros((cfg.n_pes, 6), dtype=int)
    R = ns.rhs(cfg, levels, delays)
    Rex = mms.evaluate(fr, cfg.n, tn)
    return [float(np.max(np.abs(R[v] - Rex[v])) / np.max(np.abs(Rex[v]))) for v in range(5)]


def _random_delays(cfg):
    return ns.delay_map(ns.Config(**{**cfg.__dict__, "seed": 17}), 50, ns.RANDOM)


@pytest.mark.parametrize("pes,delays_fn", [((1, 1, 1), None), ((2, 2, 2), None),
                                           ((2, 2, 2), _random_delays)],
                         ids=["one-PE", "2x2x2-sync", "2x2x2-random"])
def test_manufactured_solution_fourth_order(pes, delays_fn):
    errs = [_mms_error(N, pes, delays_fn) for N in (16, 32, 64)]
    for v in range(5):
        o1 = math.log2(errs[0][v] / errs[1][v])
        o2 = math.log2(errs[1][v] / errs[2][v])
        assert o2 > 3.5 and o1 > 3.0, (v, errs, o1, o2)
    assert max(errs[2]) < 5e-5


def _mixed_field_orders():
    """Orders (32 -> 64) on the field set whose mixed viscous terms are
    nonzero, 2x2x2 PEs, random delays.  (In the default set each du_k/dx_k
    depends on x_k alone, so the mixed terms vanish and the checks above do not
    see the mixed rule.)"""
    fc, fr = mms.exact(GAMMA, PR, MU0, OMEGA, mixed=True)
    errs = []
    for N in (16, 32, 64):
        cfg = _cfg(N, (2, 2, 2))
        dt = 0.5 * (2 * math.pi / N) ** 2
        levels = [mms.evaluate(fc, cfg.n, 0.4 - l * dt) for l in range(cfg.n_levels)]
        R = ns.rhs(cfg, levels, _random_delays(cfg))
        Rex = mms.evaluate(fr, cfg.n, 0.4)
        errs.append([float(np.max(np.abs(R[v] - Rex[v])) / np.max(np.abs(Rex[v]))) for v in range(5)])
    return [math.log2(errs[1][v] / errs[2][v]) for v in range(5)], errs


def test_manufactured_solution_with_mixed_terms_fourth_order():
    orders, errs = _mixed_field_orders()
    assert min(orders) > 3.5, (orders, errs)


def test_mixed_rule_one_sided_order_is_seen(monkeypatch):
    """The three-step rule's one-sided stencils planted as 2nd-order ones
    ((-3, 4, -1)/2 at the first point, (-1, 0, 1)/2 at the second): the
    momentum orders on the mixed field fall to about 3.15 (on the default field
    they stay at 3.98)."""
    from oracle import stencils

    def second_order(self, li, nloc):
        rows = (((0, -18.0), (1, 24.0), (2, -6.0)), ((-1, -6.0), (1, 6.0)))   # over the denominator 12
        if li < self.M:
            return rows[li]
        if li >= nloc - self.M:
            return tuple((-o, -c) for o, c in rows[nloc - 1 - li])
        return self.d1

    monkeypatch.setattr(stencils.Scheme, "one_sided", second_order)
    orders, errs = _mixed_field_orders()
    assert min(orders) < 3.4, (orders, errs)


def test_manufactured_solution_detects_dropped_term(monkeypatch):
    """Removing the viscous heating sigma_ij S_ij from the oracle breaks the
    energy-equation convergence (guards the test's own sensitivity)."""
    orig = ns.rhs

    def broken(cfg, levels, delays, fhat=None, return_aux=False):
        R, aux = orig(cfg, levels, delays, fhat, True)
        R = R.copy()
        R[4] -= aux["sigS"]
        return (R, aux) if return_aux else R

    monkeypatch.setattr(ns, "rhs", broken)
    e = _mms_error(32, (1, 1, 1))
    assert e[4] > 1e-3


def _turb_state(N, seed=2):
    return synth.initial_state((N, N, N), k0=3.0, mach_t=0.3, seed=seed, gamma=GAMMA)


@pytest.mark.parametrize("mode", [ns.SYNC, ns.PERIODIC])
def test_mass_conserved_without_delay_error(mode):
    cfg = _cfg(16, (2, 2, 2), mu0=0.03)
    U = _turb_state(16)
    run = ns.Run.start(cfg, U, mode)
    R = run.rhs()
    assert abs(R[0].sum()) < 1e-12 * np.abs(R[0]).sum() * 10


def test_euler_limit_conserves_everything():
    cfg = _cfg(16, (2, 2, 2), mu0=0.0)
    U = _turb_state(16)
    R = ns.rhs(cfg, [U] * cfg.n_levels, np.zeros((cfg.n_pes, 6), dtype=int))
    for v in range(5):
        assert abs(R[v].sum()) < 1e-12 * (np.abs(R[v]).sum() + 1.0)


def test_zero_delay_reduces_to_single_pe_euler():
    U = _turb_state(16)
    a = _cfg(16, (2, 2, 2), mu0=0.0)
    b = _cfg(16, (1, 1, 1), mu0=0.0)
    hist = synth.history(U, a.n_levels, eps=1e-2)
    Ra = ns.rhs(a, hist, np.zeros((a.n_pes, 6), dtype=int))
    Rb = ns.rhs(b, hist, np.zeros((1, 6), dtype=int))
    assert np.array_equal(Ra, Rb)


def test_zero_delay_viscous_differs_only_by_mixed_rule():
    """With viscosity, 2x2x2 PEs at k = 0 differ from one PE only through the
    one-sided mixed derivatives at PE-boundary points, so interior points agree
    exactly up to rounding."""
    U = _turb_state(16)
    a = _cfg(16, (2, 2, 2))
    b = _cfg(16, (1, 1, 1))
    Ra = ns.rhs(a, [U] * a.n_levels, np.zeros((a.n_pes, 6), dtype=int))
    Rb = ns.rhs(b, [U] * b.n_levels, np.zeros((1, 6), dtype=int))
    li = np.arange(16) % 8
    core = (li >= 2) & (li <= 5)         # the 5-point stencil fits inside the PE
    sel = core[:, None, None] & core[None, :, None] & core[None, None, :]
    assert np.array_equal(Ra[:, sel], Rb[:, sel])
    assert not np.allclose(Ra, Rb, rtol=0, atol=1e-9 * np.abs(Rb).max())


def test_kinetic_energy_budget():
    """dK/dt = <p theta> - <sigma S> + <rho f.u> (Eq. (meantke)), from the RHS."""
    fc, _ = mms.exact(GAMMA, PR, MU0, OMEGA)
    errs = []
    for N in (16, 32, 64):
        cfg = _cfg(N, (1, 1, 1))
        U = mms.evaluate(fc, cfg.n, 0.4)
        R, aux = ns.rhs(cfg, [U] * cfg.n_levels, np.zeros((1, 6), dtype=int), return_aux=True)
        vel, rho = aux["vel"], aux["rho"]
        u2 = sum(v * v for v in vel)
        dK = np.mean(sum(vel[i] * R[1 + i] for i in range(3)) - 0.5 * u2 * R[0])
        budget = np.mean(aux["p"] * aux["theta"]) - np.mean(aux["sigS"])
        errs.append(abs(dK - budget))
    assert errs[2] < errs[1] / 8 < errs[0] / 64, errs


def test_forced_budget_includes_forcing_power():
    cfg = _cfg(16, (1, 1, 1), forcing=True, kf=2.0, f_amp=0.1, f_tcorr=0.5, f_seed=3, dt=0.01)
    U = _turb_state(16)
    fh = ns.forcing_coefficients(cfg, 4)
    R0, a0 = ns.rhs(cfg, [U] * cfg.n_levels, np.zeros((1, 6), dtype=int), None, True)
    R1, a1 = ns.rhs(cfg, [U] * cfg.n_levels, np.zeros((1, 6), dtype=int), fh, True)
    vel, rho = a1["vel"], a1["rho"]
    u2 = sum(v * v for v in vel)
    dK = lambda R: np.mean(sum(vel[i] * R[1 + i] for i in range(3)) - 0.5 * u2 * R[0])
    power = np.mean(rho * sum(a1["f"][i] * vel[i] for i in range(3)))
    assert abs(power) > 1e-6
    assert abs((dK(R1) - dK(R0)) - power) < 1e-12 * (1 + abs(power))
    # forcing adds rho f_i u_i to the energy equation and rho f_i to momentum
    assert np.allclose(R1[4] - R0[4], rho * sum(a1["f"][i] * vel[i] for i in range(3)), atol=1e-13)
    assert np.array_equal(R1[0], R0[0])


@pytest.mark.parametrize("pes", [(2, 2, 2), (3, 1, 2)])
def test_brute_force_pointwise_matches_vectorised(pes):
    N = 12
    cfg = _cfg(N, pes, forcing=True, kf=2.0, f_amp=0.05, f_tcorr=0.5, dt=0.01, f_seed=9)
    U = _turb_state(N, seed=4)
    hist = synth.history(U, cfg.n_levels, eps=2e-2)
    delays = ns.delay_map(ns.Config(**{**cfg.__dict__, "seed": 5}), 30, ns.RANDOM)
    fh = ns.forcing_coefficients(cfg, 3)
    R = ns.rhs(cfg, hist, delays, fh)
    po = PointOracle(cfg, lambda l: hist[l], delays, fh, ns.forcing_modes(cfg.kf))
    rng = np.random.default_rng(0)
    pts = [tuple(int(v) for v in rng.integers(0, N, 3)) for _ in range(60)]
    pts += [(0, 0, 0), (N - 1, N - 1, N - 1), (1, 5, 6), (5, 6, 1), (6, 0, 11)]
    scale = np.abs(R).max(axis=(1, 2, 3))
    for (x, y, z) in pts:
        r = po.rhs((x, y, z))
        for v in range(5):
            assert abs(r[v] - R[v, z, y, x]) <= 1e-13 * scale[v], (x, y, z, v)


# --------------------------------------------------------------------------
# The other reading of Table B's extrapolation: q(sum_l w_l U^{n-k-l})
# --------------------------------------------------------------------------
def _xcfg(cfg):
    return ns.Config(**{**cfg.__dict__, "extrapolate_state": True})


def test_extrapolate_state_equals_default_without_delays():
    # k = 0 has weights (1, 0, ..): both readings take level n, bit for bit
    N = 16
    cfg = _cfg(N, (2, 2, 2))
    hist = synth.history(_turb_state(N, seed=3), cfg.n_levels, eps=2e-2)
    d = ns.delay_map(cfg, 40, ns.SYNC)
    assert np.array_equal(ns.rhs(cfg, hist, d), ns.rhs(_xcfg(cfg), hist, d))


def test_extrapolate_state_linear_quantities_agree():
    # The continuity fluxes rho u_d are the state's own components, linear in
    # U, so both readings give the same R_rho up to rounding; the nonlinear
    # fluxes differ at the size of the extrapolation error.
    N = 16
    cfg = _cfg(N, (2, 2, 2))
    hist = synth.history(_turb_state(N, seed=3), cfg.n_levels, eps=2e-2)
    d = _random_delays(cfg)
    a, b = ns.rhs(cfg, hist, d), ns.rhs(_xcfg(cfg), hist, d)
    assert np.max(np.abs(a[0] - b[0])) <= 1e-12 * np.max(np.abs(a[0]))
    assert np.max(np.abs(a[4] - b[4])) > 1e-9 * np.max(np.abs(a[4]))


def test_extrapolate_state_steady_history_is_exact():
    # All levels equal: the weights sum to one, so the extrapolated state is
    # the state and both readings coincide with the synchronous RHS.
    N = 16
    cfg = _cfg(N, (2, 2, 2))
    U = _turb_state(N, seed=5)
    hist = [U.copy() for _ in range(cfg.n_levels)]
    d = _random_delays(cfg)
    sync = ns.rhs(cfg, hist, np.zeros_like(d))
    scale = np.abs(sync).max(axis=(1, 2, 3))[:, None, None, None]
    assert np.max(np.abs(ns.rhs(_xcfg(cfg), hist, d) - sync) / scale) < 1e-12


def _xstate_mms_orders():
    fc, fr = mms.exact(GAMMA, PR, MU0, OMEGA)
    errs = []
    for N in (16, 32, 64):
        cfg = _xcfg(_cfg(N, (2, 2, 2)))
        dt = 0.5 * (2 * math.pi / N) ** 2
        levels = [mms.evaluate(fc, cfg.n, 0.4 - l * dt) for l in range(cfg.n_levels)]
        R = ns.rhs(cfg, levels, _random_delays(cfg))
        Rex = mms.evaluate(fr, cfg.n, 0.4)
        errs.append([float(np.max(np.abs(R[v] - Rex[v])) / np.max(np.abs(Rex[v]))) for v in range(5)])
    return [(math.log2(errs[0][v] / errs[1][v]), math.log2(errs[1][v] / errs[2][v])) for v in range(5)], errs


def test_extrapolate_state_manufactured_solution_fourth_order():
    orders, errs = _xstate_mms_orders()
    for v, (o1, o2) in enumerate(orders):
        assert o2 > 3.5 and o1 > 3.0, (v, errs, o1, o2)


def test_extrapolate_state_manufactured_solution_detects_unextrapolated_levels(monkeypatch):
    """With Table B's weights replaced by (1, 0, 0) -- the delayed level taken
    as it is, no extrapolation -- the reading's error is O(k dt) = O(dx^2) and
    the 4th-order check above fails (guards its sensitivity to the weights)."""
    from oracle import stencils
    monkeypatch.setattr(stencils, "at_weights", lambda k: (1.0, 0.0, 0.0))
    orders, errs = _xstate_mms_orders()
    assert any(o2 < 3.0 for _, o2 in orders), (orders, errs)


@pytest.mark.parametrize("pes,energy", [((2, 2, 2), ns.ENERGY_TOTAL), ((3, 1, 2), ns.ENERGY_INTERNAL)])
def test_extrapolate_state_brute_force_pointwise(pes, energy):
    N = 12
    cfg = _xcfg(_cfg(N, pes, energy_form=energy))
    U = _turb_state(N, seed=4)
    hist = synth.history(U, cfg.n_levels, eps=2e-2)
    delays = ns.delay_map(ns.Config(**{**cfg.__dict__, "seed": 5}), 30, ns.RANDOM)
    R = ns.rhs(cfg, hist, delays)
    po = PointOracle(cfg, lambda l: hist[l], delays)
    rng = np.random.default_rng(1)
    pts = [tuple(int(v) for v in rng.integers(0, N, 3)) for _ in range(40)]
    pts += [(0, 0, 0), (N - 1, N - 1, N - 1), (1, 5, 6), (5, 6, 1)]
    scale = np.abs(R).max(axis=(1, 2, 3))
    for (x, y, z) in pts:
        r = po.rhs((x, y, z))
        for v in range(5):
            assert abs(r[v] - R[v, z, y, x]) <= 1e-13 * scale[v], (x, y, z, v)
