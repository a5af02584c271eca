"""Pins of the oracle's delay map, forcing, AB2 update, statistics and of the
seeded input generator.

* delay map (Sec. 3.1, Algorithms 1 and 2): zero during the L + T_l
  synchronous start-up steps and in synchronous mode; periodic delays cycle
  0..c_r-1 with an exactly uniform histogram (Fig. del_pdf(d)); random delays
  are bounded by L and uniform (chi-square), independent per PE face;
  ordered random delays follow k_n = min(d_n, k_{n-1} + 1) (messages arrive
  in order, Alg. 1);
* forcing (Sec. 4.2): coefficients orthogonal to their wavevector, the field
  real, divergence-free and supported on |kappa| <= kappa_f; the OU variance is
  stationary;
* AB2 (Eq. (time_ab), T = 2): second-order convergence on y' = lambda y;
* statistics: closed forms on a single shear wave;
* input generator: solenoidal, zero-mean velocity with the requested M_t.
"""
import math

import numpy as np
import pytest

from oracle import ns
from paper_2003_10561_gb300 import synth


def test_delay_startup_and_sync():
    cfg = ns.Config(n=(16, 16, 16), pes=(2, 2, 2), max_delay=3, comm_period=4, seed=1)
    for n in range(cfg.n_levels):
        for mode in (ns.SYNC, ns.PERIODIC, ns.RANDOM):
            assert not ns.delay_map(cfg, n, mode).any()
    for n in range(cfg.n_levels, 40):
        assert not ns.delay_map(cfg, n, ns.SYNC).any()


def test_periodic_delays_cycle_uniformly():
    cfg = ns.Config(n=(16, 16, 16), pes=(2, 2, 2), max_delay=2, comm_period=3)
    n0 = cfg.n_levels
    seq = [int(ns.delay_map(cfg, n, ns.PERIODIC)[0, 0]) for n in range(n0, n0 + 30)]
    assert seq[:6] == [0, 1, 2, 0, 1, 2]
    counts = np.bincount(seq, minlength=3)
    assert (counts == 10).all()
    # same on every face of every PE (Sec. 3.1.2)
    m = ns.delay_map(cfg, n0 + 7, ns.PERIODIC)
    assert (m == m[0, 0]).all()


def test_random_delays_bounded_uniform_independent():
    cfg = ns.Config(n=(32, 32, 32), pes=(4, 4, 4), max_delay=2, seed=12345)
    maps = np.stack([ns.delay_map(cfg, n, ns.RANDOM) for n in range(cfg.n_levels, cfg.n_levels + 200)])
    assert maps.min() == 0 and maps.max() == 2
    counts = np.bincount(maps.ravel(), minlength=3).astype(float)
    expected = maps.size / 3.0
    chi2 = float(((counts - expected) ** 2 / expected).sum())
    assert chi2 < 13.8        # 2 dof, p = 0.001
    # neighbouring faces / PEs / steps are not copies of each other
    assert not np.array_equal(maps[0, :, 0], maps[0, :, 1])
    assert not np.array_equal(maps[0], maps[1])
    # a pure function of (seed, step, PE, face)
    assert np.array_equal(ns.delay_map(cfg, 77, ns.RANDOM), ns.delay_map(cfg, 77, ns.RANDOM))
    other = ns.Config(**{**cfg.__dict__, "seed": 54321})
    assert not np.array_equal(ns.delay_map(other, 77, ns.RANDOM), ns.delay_map(cfg, 77, ns.RANDOM))


def test_random_delay_uses_philox_word0():
    from oracle.philox import philox4x32_10, split_seed
    cfg = ns.Config(n=(8, 8, 8), pes=(2, 2, 2), max_delay=3, seed=0xDEADBEEF12345678)
    n, p, f = 41, 5, 3
    k0, k1 = split_seed(cfg.seed)
    w0 = int(philox4x32_10(n, p, f, 0x4154, k0, k1)[0])
    assert ns.delay_map(cfg, n, ns.RANDOM)[p, f] == (w0 * 4) >> 32


@pytest.mark.parametrize("L", [0, 1, 2, 4])
def test_ordered_random_delays_follow_the_arrival_recursion(L):
    """Ordered random delays (a PE's messages arrive in order, Alg. 1): the
    closed form equals the recursion k_n = min(d_n, k_{n-1} + 1) iterated step
    by step from k = 0 at the end of the start-up, with d the draws of the
    random mode; hence k never grows by more than one per step, never exceeds
    the step's draw or L, is zero through the start-up, and is identically
    zero for L = 0.  It still reaches L (a message late L steps)."""
    cfg = ns.Config(n=(24, 24, 24), pes=(3, 3, 2), max_delay=L, seed=2024)
    n0 = cfg.n_levels
    k = np.zeros((cfg.n_pes, 6), dtype=np.int64)       # k_{n0 - 1}
    seen_max = 0
    for n in range(n0 + 300):
        got = ns.delay_map(cfg, n, ns.ORDERED)
        if n < n0:
            assert not got.any()
            continue
        d = ns.delay_map(cfg, n, ns.RANDOM)
        k = np.minimum(d, k + 1)
        assert np.array_equal(got, k), n
        assert (got <= d).all() and (got >= 0).all() and (got <= L).all()
        seen_max = max(seen_max, int(got.max()))
    assert seen_max == L
    # a pure function of (seed, step, PE, face): a late step without its past
    assert np.array_equal(ns.delay_map(cfg, 2 ** 31 + 7, ns.ORDERED), ns.delay_map(cfg, 2 ** 31 + 7, ns.ORDERED))


def test_forcing_modes_shell():
    modes = ns.forcing_modes(2.0)
    assert len(modes) == 16
    full = set(modes) | {(-a, -b, -c) for a, b, c in modes}
    assert len(full) == 32
    assert all(0 < a * a + b * b + c * c <= 4 for a, b, c in full)


def test_forcing_field_solenoidal_real_band_limited():
    cfg = ns.Config(n=(16, 16, 16), forcing=True, kf=2.0, f_amp=0.3, f_tcorr=0.7, f_seed=11, dt=0.05)
    fh = ns.forcing_coefficients(cfg, 5)
    modes = np.array(ns.forcing_modes(cfg.kf), dtype=float)
    assert np.max(np.abs(np.sum(modes * fh, axis=1))) < 1e-15
    f = ns.forcing_field(cfg, fh)
    F = [np.fft.fftn(c) for c in f]
    k = np.fft.fftfreq(16, 1.0 / 16)
    KZ, KY, KX = np.meshgrid(k, k, k, indexing="ij")
    div = 1j * (KX * F[0] + KY * F[1] + KZ * F[2])
    assert np.max(np.abs(div)) < 1e-10 * np.max(np.abs(F[0]))
    k2 = KX ** 2 + KY ** 2 + KZ ** 2
    for c in range(3):
        assert np.max(np.abs(F[c][k2 > 4.0 + 1e-9])) < 1e-10 * np.max(np.abs(F[c]))
        assert np.max(np.abs(F[c][k2 == 0])) < 1e-10 * np.max(np.abs(F[c]))


def test_forcing_ou_stationary_variance():
    cfg = ns.Config(n=(8, 8, 8), forcing=True, kf=2.0, f_amp=1.0, f_tcorr=0.2, f_seed=2, dt=0.05)
    modes = ns.forcing_modes(cfg.kf)
    a = math.exp(-cfg.dt / cfg.f_tcorr)
    b = math.sqrt(1 - a * a)
    fh = ns.solenoidal_projection(modes, ns.forcing_noise(cfg, 0, modes))
    acc = []
    for s in range(1, 1500):
        fh = a * fh + b * ns.solenoidal_projection(modes, ns.forcing_noise(cfg, s, modes))
        acc.append(np.mean(np.abs(fh) ** 2))
    # re and im each unit variance per component, projection keeps 2 of 3 dims
    assert abs(np.mean(acc) - 2.0 * 2.0 / 3.0) < 0.1
    # the recursion in forcing_coefficients is the same process
    ref = ns.forcing_coefficients(cfg, 3)
    fh = cfg.f_amp * ns.solenoidal_projection(modes, ns.forcing_noise(cfg, 0, modes))
    for s in range(1, 4):
        fh = a * fh + cfg.f_amp * b * ns.solenoidal_projection(modes, ns.forcing_noise(cfg, s, modes))
    assert np.allclose(ref, fh, rtol=0, atol=1e-15)


def test_ab2_second_order():
    lam = -1.3 + 0.7j
    errs = []
    for nsteps in (50, 100, 200):
        h = 1.0 / nsteps
        y, fprev = np.array([1.0 + 0j]), None
        for _ in range(nsteps):
            f = lam * y
            y = ns.ab2_update(y, f, fprev, h)
            fprev = f
        errs.append(abs(y[0] - np.exp(lam)))
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(1.9 < o < 2.1 for o in orders), orders


def test_statistics_shear_wave():
    """u = a sin(y): eps = mu <(du/dy)^2>, Omega = <(du/dy)^2>, K = rho a^2/4."""
    N = 32
    cfg = ns.Config(n=(N, N, N), mu0=0.01, visc_exp=0.0)
    y = np.arange(N) * 2 * math.pi / N
    a = 0.1
    U = np.zeros((5, N, N, N))
    U[0] = 1.0
    U[1] = a * np.sin(y)[None, :, None]
    U[4] = (1.0 / cfg.gamma) / (cfg.gamma - 1) + 0.5 * U[1] ** 2
    R, aux = ns.rhs(cfg, [U] * cfg.n_levels, np.zeros((1, 6), dtype=int), return_aux=True)
    st = ns.statistics(cfg, U, aux)
    h = cfg.dx[1]
    k1 = (8 * math.sin(h) - math.sin(2 * h)) / (6 * h)       # modified wavenumber
    g2 = 0.5 * (a * k1) ** 2                                 # <(du/dy)^2>
    assert abs(st["dissipation"] - cfg.mu0 * g2) < 1e-15
    assert abs(st["enstrophy"] - g2) < 1e-14
    assert abs(st["tke"] - a * a / 4) < 1e-15
    assert abs(st["grad_m2"]) < 1e-30
    assert abs(st["mass"] - 1.0) < 1e-15
    assert abs(st["max_wave_speed"] - (a + 1.0)) < 1e-12
    assert abs(st["min_p"] - 1 / cfg.gamma) < 1e-15


def test_dt_from_cfl():
    N = 16
    cfg = ns.Config(n=(N, N, N))
    U = synth.initial_state((N, N, N), mach_t=0.3, seed=0)
    dt = ns.dt_from_cfl(cfg, U, 0.5)
    s = ns.max_wave_speed(cfg, U)
    assert abs(dt - 0.5 * cfg.dx[0] / s) < 1e-15


def test_synth_initial_state():
    n = (24, 24, 24)
    U = synth.initial_state(n, k0=4.0, mach_t=0.3, seed=7)
    vel = U[1:4] / U[0]
    assert abs(math.sqrt(np.mean((vel ** 2).sum(axis=0))) - 0.3) < 1e-12
    assert np.max(np.abs(vel.mean(axis=(1, 2, 3)))) < 1e-15
    k = np.fft.fftfreq(24, 1.0 / 24)
    KZ, KY, KX = np.meshgrid(k, k, k, indexing="ij")
    F = [np.fft.fftn(vel[c]) for c in range(3)]
    div = KX * F[0] + KY * F[1] + KZ * F[2]
    assert np.max(np.abs(div)) < 1e-10 * np.max(np.abs(F[0]))
    assert np.array_equal(U, synth.initial_state(n, k0=4.0, mach_t=0.3, seed=7))
    assert not np.array_equal(U, synth.initial_state(n, k0=4.0, mach_t=0.3, seed=8))
    p = (1.4 - 1) * (U[4] - 0.5 * U[0] * (vel ** 2).sum(axis=0))
    assert np.allclose(p, 1 / 1.4, rtol=0, atol=1e-14)
