"""GPU parity of the paper-faithful variants: the internal-energy form
(Eq. (ie), fifth variable rho e) and Sutherland's viscosity law, on both
kernel paths and in both orders, against the FP64 oracle.  Bars as for the
default form: FP64 RHS <= 1e-12, 60 AB2 steps <= 1e-10, FP32 RHS <= 2e-4
(3e-4 at 6th order), statistics <= 1e-11."""
import numpy as np
import pytest

from oracle import ns
from paper_2003_10561_gb300 import synth
from tests.test_gpu_parity import GAMMA, OMEGA, PR, PATHS, lib, make, ocfg, rel_linf  # noqa: F401

pytestmark = pytest.mark.gpu

VARIANTS = {
    "rhoe": dict(energy_form=ns.ENERGY_INTERNAL, visc_law=ns.VISC_POWER),
    "sutherland": dict(energy_form=ns.ENERGY_TOTAL, visc_law=ns.VISC_SUTHERLAND),
    "rhoe-sutherland": dict(energy_form=ns.ENERGY_INTERNAL, visc_law=ns.VISC_SUTHERLAND),
}


def to_form(cfg, levels):
    """The same flow with the configuration's fifth variable."""
    if cfg.energy_form == ns.ENERGY_TOTAL:
        return levels
    out = []
    for lv in levels:
        _, _, p, _ = ns.primitives(ns.Config(n=cfg.n, gamma=cfg.gamma), lv)
        out.append(np.stack([lv[0], lv[1], lv[2], lv[3], p / (cfg.gamma - 1.0)]))
    return np.stack(out)


def lib_kw(v):
    return dict(energy_form=v["energy_form"], visc_law=v["visc_law"], sutherland_s=0.368)


@pytest.mark.parametrize("kf", [2.0, 3.0])
@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("name", list(VARIANTS))
def test_rhs_parity_fp64_variants(lib, name, path, kf):
    """Each variant forced on the workload's shell (kappa_f = 2) and on the
    paper's (kappa_f = 3, Sec. 4.2)."""
    v = VARIANTS[name]
    n, pes = (16, 16, 16), (2, 2, 2)
    kw = dict(mu0=0.02, dt=2e-3, max_delay=2, seed=77, forcing=1, kf=kf, f_amp=0.1, f_tcorr=0.5, f_seed=4)
    c = ocfg(n, pes, **{**kw, "forcing": True}, **v, suth_s=0.368)
    U0 = synth.initial_state(n, k0=3.0, mach_t=0.3, seed=11)
    hist = to_form(c, synth.history(U0, c.n_levels, eps=2e-2, seed=5))
    s = make(lib, n, pes, path=path, **kw, **lib_kw(v))
    s.set_history(hist, 9)
    R = s.rhs("random")
    Rref = ns.rhs(c, hist, ns.delay_map(c, 9, ns.RANDOM), ns.forcing_coefficients(c, 9))
    assert max(rel_linf(R, Rref)) <= 1e-12, rel_linf(R, Rref)


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("omega", [0.76, 0.5, 0.7, 1.0, 0.0, 0.7123456789])
def test_rhs_parity_fp64_power_law_exponents(lib, omega, path):
    """The power law mu0 T^omega for exponents that are fractions p/q with
    q <= 64 (0.76 = 19/25, 1/2, 7/10, 1, 0: the FP64 kernels take the
    root-correction form) and one that is not (the exponential form), on a
    field whose temperature spans a wide range (T from about 0.3 to 3)."""
    n, pes = (16, 16, 16), (2, 2, 2)
    kw = dict(mu0=0.02, dt=2e-3, max_delay=2, seed=77, visc_exp=omega)
    c = ocfg(n, pes, **kw)
    U0 = synth.initial_state(n, k0=3.0, mach_t=0.3, seed=11)
    x = np.arange(n[0]) * 2 * np.pi / n[0]
    U0 = U0.copy()
    # E raised and lowered along x: T = gamma (gamma - 1) (E - K) / rho
    K = 0.5 * (U0[1] ** 2 + U0[2] ** 2 + U0[3] ** 2) / U0[0]
    U0[4] = K + (U0[4] - K) * (1.0 + 0.82 * np.sin(x))[None, None, :] * 1.6
    hist = synth.history(U0, c.n_levels, eps=2e-2, seed=5)
    _, _, _, T = ns.primitives(c, hist[0])
    assert T.min() < 0.5 and T.max() > 2.5
    s = make(lib, n, pes, path=path, **kw)
    s.set_history(hist, 9)
    R = s.rhs("random")
    Rref = ns.rhs(c, hist, ns.delay_map(c, 9, ns.RANDOM))
    assert max(rel_linf(R, Rref)) <= 1e-12, rel_linf(R, Rref)


@pytest.mark.parametrize("prec", ["p32", "p32c"])
@pytest.mark.parametrize("path", PATHS)
def test_rhs_parity_fp32_variant(lib, path, prec):
    v = VARIANTS["rhoe-sutherland"]
    n, pes = (16, 16, 16), (2, 2, 2)
    kw = dict(mu0=0.02, dt=2e-3, max_delay=2, seed=77)
    c = ocfg(n, pes, **kw, **v, suth_s=0.368)
    U0 = synth.initial_state(n, k0=3.0, mach_t=0.3, seed=11)
    hist = to_form(c, synth.history(U0, c.n_levels, eps=2e-2, seed=5))
    s = make(lib, n, pes, prec, path=path, **kw, **lib_kw(v))
    s.set_history(hist, 9)
    R = s.rhs("random")
    Rref = ns.rhs(c, hist, ns.delay_map(c, 9, ns.RANDOM))
    assert max(rel_linf(R, Rref)) <= 2e-4, rel_linf(R, Rref)


@pytest.mark.parametrize("path", PATHS)
def test_steps_parity_fp64_variant(lib, path):
    """60 AB2 steps of the internal-energy form with Sutherland viscosity and
    random delays, from a state through the synchronous start-up."""
    v = VARIANTS["rhoe-sutherland"]
    n, pes = (16, 16, 16), (2, 2, 2)
    kw = dict(mu0=0.03, dt=4e-3, max_delay=2, seed=5)
    c = ocfg(n, pes, **kw, **v, suth_s=0.368)
    U0 = to_form(c, [synth.initial_state(n, k0=3.0, mach_t=0.3, seed=21)])[0]
    s = make(lib, n, pes, path=path, **kw, **lib_kw(v))
    s.set_state(U0)
    run = ns.Run.start(c, U0, ns.RANDOM)
    for _ in range(60):
        run.step()
    s.step(60, "random")
    assert max(rel_linf(s.get_state(), run.levels[0])) <= 1e-10


def test_stats_and_order6_variant(lib):
    """Statistics of the internal-energy form, and the 6th-order scheme with
    both variants (multi-pass path)."""
    v = VARIANTS["rhoe-sutherland"]
    n, pes = (28, 28, 28), (2, 2, 2)
    kw = dict(mu0=0.02, dt=1e-3, max_delay=2, seed=1)
    for order in (4, 6):
        c = ocfg(n, pes, order=order, **kw, **v, suth_s=0.368)
        U0 = synth.initial_state(n, k0=4.0, mach_t=0.3, seed=13)
        hist = to_form(c, synth.history(U0, c.n_levels, eps=1e-2, seed=2))
        s = make(lib, n, pes, order=order, **kw, **lib_kw(v))
        s.set_history(hist, 11)
        R = s.rhs("random")
        Rref, aux = ns.rhs(c, hist, ns.delay_map(c, 11, ns.RANDOM), None, True)
        assert max(rel_linf(R, Rref)) <= 1e-12, (order, rel_linf(R, Rref))
        st = s.stats()
        ref = ns.statistics(c, hist[0], aux)
        for k in ("energy", "tke", "dissipation", "pressure_dilatation", "min_p", "max_wave_speed"):
            assert abs(st[k] - ref[k]) <= 1e-11 * abs(ref[k]) + 1e-15, (order, k, st[k], ref[k])
        s.close()
