"""Pins of the oracle's paper-faithful variants (Sec. 2):

* the internal-energy form, Eq. (ie) -- fifth variable rho e -- and
  Sutherland's viscosity law converge at 4th order to the sympy-exact
  right-hand side of the same PDEs (with one PE and with 2x2x2 PEs under
  random delays);
* the two energy forms describe the same flow: for one state, the total
  energy rate equals the internal energy rate plus the kinetic energy rate
  u_i R_{rho u_i} - |u|^2/2 R_rho, up to 4th-order truncation;
* momentum and mass right-hand sides do not depend on the form;
* the brute-force pointwise evaluation equals the vectorised one.
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
    base = dict(n=(N, N, N), pes=pes, gamma=GAMMA, prandtl=PR, mu0=MU0, visc_exp=OMEGA, max_delay=2, seed=17)
    base.update(kw)
    return ns.Config(**base)


def _mms_error(N, pes, internal, suth, random):
    fc, fr = mms.exact(GAMMA, PR, MU0, OMEGA, internal, 0.368 if suth else None)
    cfg = _cfg(N, pes, energy_form=ns.ENERGY_INTERNAL if internal else ns.ENERGY_TOTAL,
               visc_law=ns.VISC_SUTHERLAND if suth else ns.VISC_POWER, suth_s=0.368)
    dt = 0.5 * (2 * math.pi / N) ** 2
    levels = [mms.evaluate(fc, cfg.n, 0.4 - l * dt) for l in range(cfg.n_levels)]
    delays = ns.delay_map(cfg, 50, ns.RANDOM) if random else np.zeros((cfg.n_pes, 6), dtype=int)
    R = ns.rhs(cfg, levels, delays)
    Rex = mms.evaluate(fr, cfg.n, 0.4)
    return [float(np.max(np.abs(R[v] - Rex[v])) / np.max(np.abs(Rex[v]))) for v in range(5)]


@pytest.mark.parametrize("internal,suth,pes,random", [
    (True, False, (1, 1, 1), False), (True, False, (2, 2, 2), True),
    (False, True, (2, 2, 2), True), (True, True, (1, 1, 1), False)],
    ids=["rhoe", "rhoe-2x2x2-random", "sutherland-2x2x2-random", "rhoe-sutherland"])
def test_manufactured_solution_fourth_order(internal, suth, pes, random):
    errs = [_mms_error(N, pes, internal, suth, random) for N in (16, 32, 64)]
    for v in range(5):
        o = math.log2(errs[1][v] / errs[2][v])
        assert o > 3.5, (v, errs, o)
    assert max(errs[2]) < 5e-5


def _states(N, seed=3):
    """The same flow as total-energy and as internal-energy state."""
    U = synth.initial_state((N, N, N), k0=3.0, mach_t=0.3, seed=seed, gamma=GAMMA)
    hist = synth.history(U, 5, eps=2e-2, seed=seed)
    tot = ns.Config(n=(N, N, N), gamma=GAMMA, mu0=MU0)
    out_t, out_i = [], []
    for lv in hist:
        rho, vel, p, T = ns.primitives(tot, lv)
        rhoe = p / (GAMMA - 1.0)
        out_t.append(lv)
        out_i.append(np.stack([lv[0], lv[1], lv[2], lv[3], rhoe]))
    return out_t, out_i


def test_energy_forms_agree_through_kinetic_energy_rate():
    """On the smooth manufactured field (the same flow at every resolution)."""
    fct, _ = mms.exact(GAMMA, PR, MU0, OMEGA, False, None)
    fci, _ = mms.exact(GAMMA, PR, MU0, OMEGA, True, None)
    errs = []
    for N in (16, 32, 64):
        Ut = [mms.evaluate(fct, (N, N, N), 0.4)] * 5
        Ui = [mms.evaluate(fci, (N, N, N), 0.4)] * 5
        ct = _cfg(N, (1, 1, 1))
        ci = _cfg(N, (1, 1, 1), energy_form=ns.ENERGY_INTERNAL)
        Rt = ns.rhs(ct, Ut, np.zeros((1, 6), dtype=int))
        Ri, aux = ns.rhs(ci, Ui, np.zeros((1, 6), dtype=int), return_aux=True)
        # mass and momentum do not depend on the form
        for v in range(4):
            assert np.allclose(Rt[v], Ri[v], rtol=0, atol=1e-11 * np.abs(Rt[v]).max())
        vel = aux["vel"]
        ke_rate = sum(vel[i] * Ri[1 + i] for i in range(3)) - 0.5 * sum(v * v for v in vel) * Ri[0]
        errs.append(np.max(np.abs(Rt[4] - (Ri[4] + ke_rate))) / np.max(np.abs(Rt[4])))
    assert errs[2] < errs[1] / 12 < errs[0] / 144, errs


def test_internal_form_dropped_pressure_work_detected():
    """Without -p theta the internal-energy RHS misses the exact one (guards
    the sensitivity of the manufactured-solution pin)."""
    N = 32
    fc, fr = mms.exact(GAMMA, PR, MU0, OMEGA, True, None)
    cfg = _cfg(N, (1, 1, 1), energy_form=ns.ENERGY_INTERNAL)
    U = mms.evaluate(fc, cfg.n, 0.4)
    R, aux = ns.rhs(cfg, [U] * cfg.n_levels, np.zeros((1, 6), dtype=int), return_aux=True)
    Rex = mms.evaluate(fr, cfg.n, 0.4)
    good = np.max(np.abs(R[4] - Rex[4]))
    bad = np.max(np.abs(R[4] + aux["p"] * aux["theta"] - Rex[4]))
    assert bad > 100 * good


@pytest.mark.parametrize("internal,suth", [(True, False), (True, True), (False, True)])
def test_brute_force_pointwise_matches_vectorised(internal, suth):
    N = 12
    cfg = _cfg(N, (2, 2, 2), energy_form=ns.ENERGY_INTERNAL if internal else ns.ENERGY_TOTAL,
               visc_law=ns.VISC_SUTHERLAND if suth else ns.VISC_POWER, forcing=True, kf=2.0, f_amp=0.05,
               f_tcorr=0.5, dt=0.01, f_seed=9, seed=5)
    Ut, Ui = _states(N, seed=4)
    hist = (Ui if internal else Ut)[:cfg.n_levels]
    delays = ns.delay_map(cfg, 30, ns.RANDOM)
    fh = ns.forcing_coefficients(cfg, 3)
    R = ns.rhs(cfg, hist, delays, fh)
    po = PointOracle(cfg, lambda l: hist[l], delays, fh, ns.forcing_modes(cfg.kf))
    rng = np.random.default_rng(1)
    pts = [tuple(int(v) for v in rng.integers(0, N, 3)) for _ in range(40)] + [(0, 0, 0), (11, 6, 5)]
    scale = np.abs(R).max(axis=(1, 2, 3))
    for (x, y, z) in pts:
        r = po.rhs((x, y, z))
        for v in range(5):
            assert abs(r[v] - R[v, z, y, x]) <= 1e-13 * scale[v], (x, y, z, v)
