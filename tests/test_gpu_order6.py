"""GPU parity of the 6th-order AT scheme (Table B rows (1,6) and (2,6),
T_l = 4, three ghost layers per PE face) against the FP64 oracle.

Same bars as the 4th-order parity tests: delay maps bit-exact (start-up now
L + 4 steps); FP64 relative L-infinity per conserved variable <= 1e-12 for
one RHS and <= 1e-10 after 60 AB2 steps; FP32-bulk <= 3e-4 per RHS (the
6th-order D2 stencil's absolute coefficients sum to 6.0/dx^2 against 5.3/dx^2
at 4th order, so the 4th-order FP32 bound of 2e-4 is scaled by that ratio
with margin).  The fused path runs the 4th-order scheme only and refuses
order 6.
"""
import numpy as np
import pytest

from oracle import ns
from oracle.pointwise import PointOracle
from paper_2003_10561_gb300 import synth
from tests.test_gpu_parity import GAMMA, OMEGA, PR, lib, ocfg, rel_linf  # noqa: F401

pytestmark = pytest.mark.gpu


def make6(lib, n, pes, precision="p64", **kw):
    return lib.Solver(n=n, pes=pes, precision=precision, gamma=GAMMA, prandtl=PR, visc_exp=OMEGA, order=6, **kw)


@pytest.mark.parametrize("mode", ["sync", "periodic", "random"])
def test_delay_map_bit_exact_order6(lib, mode):
    s = make6(lib, (28, 21, 14), (4, 3, 2), mu0=0.01, dt=1e-3, max_delay=3, comm_period=4, seed=99)
    c = ocfg((28, 21, 14), (4, 3, 2), max_delay=3, comm_period=4, seed=99, order=6)
    for step in (0, 6, 7, 8, 13, 1000):
        ref = ns.delay_map(c, step, lib.MODES[mode])
        assert np.array_equal(s.delay_map(step, mode).astype(np.int64), ref), (mode, step)
    assert s.info()["n_levels"] == 7 and s.info()["order"] == 6


CASES6 = [
    # n, pes, mode, step, L
    ((32, 32, 32), (1, 1, 1), "sync", 0, 2),
    ((14, 14, 14), (2, 2, 2), "random", 10, 2),
    ((14, 14, 14), (2, 2, 2), "periodic", 9, 2),
    ((21, 14, 28), (3, 2, 4), "random", 12, 3),    # 7-point PEs: every point is a face point
    ((32, 16, 24), (4, 1, 3), "random", 13, 4),    # a direction without faces, PEs 8 x 16 x 8
    ((30, 20, 18), (3, 2, 2), "periodic", 8, 2),   # PEs 10 x 10 x 9
]


@pytest.mark.parametrize("n,pes,mode,step,L", CASES6)
def test_rhs_parity_fp64_order6(lib, n, pes, mode, step, L):
    U0 = synth.initial_state(n, k0=3.0, mach_t=0.3, seed=11)
    kw = dict(mu0=0.02, dt=2e-3, max_delay=L, comm_period=L + 1, seed=77)
    c = ocfg(n, pes, order=6, **kw)
    hist = synth.history(U0, c.n_levels, eps=2e-2, seed=5)
    s = make6(lib, n, pes, **kw)
    s.set_history(hist, step)
    R = s.rhs(mode)
    Rref = ns.rhs(c, hist, ns.delay_map(c, step, lib.MODES[mode]))
    assert max(rel_linf(R, Rref)) <= 1e-12, rel_linf(R, Rref)


def test_rhs_parity_fp64_order6_forced(lib):
    n, pes = (14, 14, 14), (2, 2, 2)
    kw = dict(mu0=0.02, dt=5e-3, max_delay=2, seed=3, forcing=1, kf=2.0, f_amp=0.2, f_tcorr=0.3, f_seed=99)
    U0 = synth.initial_state(n, k0=3.0, mach_t=0.3, seed=12)
    c = ocfg(n, pes, order=6, **{**kw, "forcing": True})
    hist = synth.history(U0, c.n_levels, eps=1e-2, seed=6)
    s = make6(lib, n, pes, **kw)
    s.set_history(hist, 9)
    R = s.rhs("random")
    Rref = ns.rhs(c, hist, ns.delay_map(c, 9, ns.RANDOM), ns.forcing_coefficients(c, 9))
    assert max(rel_linf(R, Rref)) <= 1e-12, rel_linf(R, Rref)


@pytest.mark.parametrize("prec", ["p32", "p32c"])
@pytest.mark.parametrize("n,pes,mode,step,L", CASES6[1:4])
def test_rhs_parity_fp32_order6(lib, n, pes, mode, step, L, prec):
    U0 = synth.initial_state(n, k0=3.0, mach_t=0.3, seed=11)
    kw = dict(mu0=0.02, dt=2e-3, max_delay=L, comm_period=L + 1, seed=77)
    c = ocfg(n, pes, order=6, **kw)
    hist = synth.history(U0, c.n_levels, eps=2e-2, seed=5)
    s = make6(lib, n, pes, prec, **kw)
    s.set_history(hist, step)
    R = s.rhs(mode)
    Rref = ns.rhs(c, hist, ns.delay_map(c, step, lib.MODES[mode]))
    assert max(rel_linf(R, Rref)) <= 3e-4, rel_linf(R, Rref)


@pytest.mark.parametrize("mode", ["random", "periodic"])
def test_at_steps_parity_fp64_order6(lib, mode):
    """14^3, 2x2x2 PEs of 7^3, from a state through the L + 4 synchronous
    start-up into delayed steps: 60 AB2 steps, the ring of past levels written
    by the step kernel itself."""
    n, pes = (14, 14, 14), (2, 2, 2)
    U0 = synth.initial_state(n, k0=3.0, mach_t=0.3, seed=21)
    kw = dict(mu0=0.03, dt=4e-3, max_delay=2, comm_period=3, seed=5)
    c = ocfg(n, pes, order=6, **kw)
    s = make6(lib, n, pes, **kw)
    s.set_state(U0)
    run = ns.Run.start(c, U0, lib.MODES[mode])
    for _ in range(60):
        run.step()
    s.step(60, mode)
    err = rel_linf(s.get_state(), run.levels[0])
    assert max(err) <= 1e-10, err


def test_stats_parity_fp64_order6(lib):
    n, pes = (28, 28, 28), (2, 2, 2)
    U0 = synth.initial_state(n, k0=4.0, mach_t=0.3, seed=13)
    c = ocfg(n, pes, mu0=0.02, dt=1e-3, max_delay=2, seed=1, order=6)
    hist = synth.history(U0, c.n_levels, eps=1e-2, seed=2)
    s = make6(lib, n, pes, mu0=0.02, dt=1e-3, max_delay=2, seed=1)
    s.set_history(hist, 11)
    s.rhs("random")
    st = s.stats()
    R, aux = ns.rhs(c, hist, ns.delay_map(c, 11, ns.RANDOM), None, True)
    ref = ns.statistics(c, hist[0], aux)
    for k in ("tke", "dissipation", "enstrophy", "grad_m2", "grad_m3", "pressure_dilatation", "max_wave_speed"):
        assert abs(st[k] - ref[k]) <= 1e-11 * abs(ref[k]) + 1e-15, (k, st[k], ref[k])


def test_full_size_sampled_parity_order6(lib):
    """192^3 with 8x8x8 PEs of 24^3, random delays L = 3 at a delayed step:
    sampled points (face, edge and corner layers included) against the
    brute-force pointwise oracle.

    Tolerance: the 4th-order full-size bound (1e-11 at L = 2) scaled by the
    rounding amplification of the AT extrapolation, sum_l |w_l(L)|: 17 for the
    4th-order weights at k = 2, 111 for the 6th-order weights at k = 3
    (20 + 45 + 36 + 10), so 1e-11 * 111 / 17 = 6.5e-11.  The kernel
    extrapolates the quantities first and applies one stencil, the oracle
    applies T_l stencils and weights them; the two orders round differently
    within that bound."""
    n, pes, L = (192, 192, 192), (8, 8, 8), 3
    U0 = synth.initial_state(n, k0=4.0, mach_t=0.3, seed=1)
    c = ocfg(n, pes, mu0=0.004, dt=1e-3, max_delay=L, seed=31, order=6)
    hist = synth.history(U0, c.n_levels, eps=1e-2, seed=3)
    step = 19
    s = make6(lib, n, pes, mu0=0.004, dt=1e-3, max_delay=L, seed=31)
    s.set_history(hist, step)
    R = s.rhs("random")
    s.close()
    po = PointOracle(c, lambda l: hist[l], ns.delay_map(c, step, ns.RANDOM))
    rng = np.random.default_rng(8)
    pts = {tuple(int(rng.integers(0, 192)) for _ in range(3)) for _ in range(60)}
    for a in (0, 1, 2, 3, 20, 21, 22, 23, 24, 25, 26):
        pts.add((a, 24 * 3 + 1, (a + 5) % 192))
        pts.add((100, a, 47))
        pts.add((191, 2, a))
    pts = sorted(pts)
    ref = np.array([po.rhs(p) for p in pts])
    got = np.array([[R[v, z, y, x] for v in range(5)] for (x, y, z) in pts])
    err = np.max(np.abs(got - ref), axis=0) / np.max(np.abs(ref), axis=0)
    assert np.max(err) <= 6.5e-11, err


def test_fused_path_refuses_order6(lib):
    with pytest.raises(lib.AtDnsError) as ei:
        make6(lib, (32, 32, 32), (2, 2, 2), path="fused", mu0=0.01, dt=1e-3)
    assert ei.value.code == lib.AT_DNS_E_UNSUPPORTED
    s = make6(lib, (32, 32, 32), (2, 2, 2), mu0=0.01, dt=1e-3)
    s.set_state(synth.initial_state((32, 32, 32), seed=1))
    best_ms = s.tune("random", trials=2)
    assert s.info()["kernel_path"] == lib.AT_DNS_PATH_MULTIPASS
    assert best_ms > 0
