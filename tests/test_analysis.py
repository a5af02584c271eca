"""Pins of the host analysis (spectra, PDFs, slices) against closed forms:
Parseval sums, single Fourier modes, exact spectral derivatives, the
Taylor-Green vortex's enstrophy and dissipation, normalised PDFs, and a
k^(-5/3) field whose compensated spectrum is flat."""
import math

import numpy as np
import pytest

from paper_2003_10561_gb300 import analysis, synth


def grid(n):
    ax = [np.arange(m) * 2 * np.pi / m for m in n]
    Z, Y, X = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    return X, Y, Z


def test_parseval_energy_and_pressure():
    U = synth.initial_state((24, 20, 16), k0=3.0, mach_t=0.3, seed=2)
    rho, vel, p, T = analysis.primitives(U)
    E = analysis.energy_spectrum(vel)
    assert abs(E.sum() - 0.5 * np.mean(vel[0] ** 2 + vel[1] ** 2 + vel[2] ** 2)) < 1e-14
    Ep = analysis.pressure_spectrum(p)
    assert abs(Ep.sum() - np.var(p)) < 1e-14 * (1 + np.var(p))


def test_single_mode_lands_in_its_shell():
    n = (16, 16, 16)
    X, Y, Z = grid(n)
    u = np.cos(3 * X + 4 * Z)          # |k| = 5
    E = analysis.energy_spectrum([u, 0 * u, 0 * u])
    assert abs(E[5] - 0.25) < 1e-15 and abs(E.sum() - 0.25) < 1e-15


@pytest.mark.parametrize("m", [1, 3, 7])
def test_spectral_gradient_exact(m):
    n = (16, 12, 20)
    X, Y, Z = grid(n)
    f = np.sin(m * X) * np.cos(2 * Y) + np.sin(3 * Z)
    g = analysis.spectral_gradient(f)
    assert np.allclose(g[0], m * np.cos(m * X) * np.cos(2 * Y), atol=1e-12)
    assert np.allclose(g[1], -2 * np.sin(m * X) * np.sin(2 * Y), atol=1e-12)
    assert np.allclose(g[2], 3 * np.cos(3 * Z), atol=1e-12)


def test_taylor_green_enstrophy_and_dissipation():
    """u = sin x cos y, v = -cos x sin y: omega_z = 2 sin x sin y, so
    <omega^2> = 1; incompressible, so <sigma S> = 2 mu <S_ij S_ij> = mu <omega^2>."""
    n = (32, 32, 8)
    X, Y, Z = grid(n)
    vel = [np.sin(X) * np.cos(Y), -np.cos(X) * np.sin(Y), 0 * X]
    A = analysis.gradients(vel)
    assert abs(analysis.enstrophy_field(A).mean() - 1.0) < 1e-13
    assert abs(analysis.dissipation_field(A, 0.01).mean() - 0.01) < 1e-15


def test_pdf_is_normalised_and_centred():
    rng = np.random.default_rng(0)
    x = rng.lognormal(0.0, 1.0, 100000)
    c, d = analysis.normalized_pdf(x, 50)
    edges = np.logspace(np.log10((x / x.mean()).min()), np.log10((x / x.mean()).max()) * (1 + 1e-12), 51)
    w = np.diff(edges)
    assert abs(np.sum(d * w) - 1.0) < 1e-12
    c2, d2 = analysis.normalized_pdf(rng.standard_normal(100000), 40, log=False)
    assert abs(np.sum(d2 * (c2[1] - c2[0])) - 1) < 1e-9


def test_compensated_spectrum_flat_for_minus_five_thirds():
    """A field whose shell energy is kappa^(-5/3) (random phases) gives a
    compensated spectrum equal to <eps>^(-2/3) on every populated shell."""
    n = (32, 32, 32)
    kx, ky, kz = analysis.wavenumbers(n)
    kmag = np.sqrt(kx * kx + ky * ky + kz * kz)
    shell = np.floor(kmag + 0.5).astype(int)
    counts = np.bincount(shell.ravel())
    rng = np.random.default_rng(3)
    phase = np.exp(2j * np.pi * rng.random(kmag.shape))
    amp = np.zeros_like(kmag)
    ok = (shell > 0) & (shell <= 10)
    amp[ok] = np.sqrt(shell[ok] ** (-5.0 / 3.0) / counts[shell[ok]] * 2.0)
    uh = amp * phase
    u = np.real(np.fft.ifftn(uh)) * uh.size
    E = analysis.energy_spectrum([u, 0 * u, 0 * u])
    k = np.arange(1, 11)
    ratio = E[1:11] / k ** (-5.0 / 3.0)
    # taking the real part halves the power evenly over +/- k pairs
    assert np.allclose(ratio / ratio.mean(), 1.0, rtol=0.35)


def test_analyze_snapshot_runs_on_both_forms():
    U = synth.initial_state((16, 16, 16), k0=3.0, mach_t=0.3, seed=5)
    a = analysis.analyze(U, mu0=0.02)
    rho, vel, p, T = analysis.primitives(U)
    Ui = U.copy()
    Ui[4] = p / 0.4
    b = analysis.analyze(Ui, mu0=0.02, energy_form=analysis.ENERGY_INTERNAL)
    assert np.allclose(a["E"], b["E"]) and np.allclose(a["Ep"], b["Ep"])
    assert a["eps"] > 0 and a["eta"] > 0 and a["re_lambda"] > 0
    assert a["enstrophy_slice"].shape == (16, 16)
    assert abs(np.mean(a["enstrophy_slice"]) - 1.0) < 0.5
    # dissipation ~ nu <omega^2> for a nearly incompressible field at rho = 1
    assert abs(a["eps"] - a["nu"] * a["enstrophy"]) < 0.2 * a["eps"]


class _FakeForced:
    """Stands in for a forced solver: the kinetic energy relaxes towards 1 as
    1 - exp(-t / 300) over the steps taken (a stationary state is approached
    from rest)."""

    def __init__(self):
        self.t = 0
        self.modes = set()

    def set_state(self, state):
        self.t = 0

    def step(self, n, mode):
        self.t += n
        self.modes.add(mode)

    def stats(self):
        return {"tke": 1.0 - math.exp(-self.t / 300.0)}

    def get_state(self):
        return ("state at step", self.t)


def test_forced_stationary_state_stops_when_block_means_settle():
    """Blocks of 200 steps: the helper stops at the first block whose mean
    kinetic energy is within 2 % of the previous block's, i.e. when the
    relaxation has decayed enough, and returns the state of that step."""
    s = _FakeForced()
    state, hist = analysis.forced_stationary_state(s, None, block=200, max_blocks=50, tol=0.02)
    assert s.modes == {"sync"}
    assert len(hist) >= 3 and abs(hist[-1] - hist[-2]) <= 0.02 * abs(hist[-2])
    assert all(abs(hist[i] - hist[i - 1]) > 0.02 * abs(hist[i - 1]) for i in range(1, len(hist) - 1))
    assert state == ("state at step", 200 * len(hist))
    # a block limit ends the search even when the energy has not settled
    s2 = _FakeForced()
    _, hist2 = analysis.forced_stationary_state(s2, None, block=10, max_blocks=4, tol=1e-9)
    assert len(hist2) == 4


def test_synth_viscosity_meets_resolution_target():
    """mu0_for_resolution: with rho = T = 1 (nu = mu0) the initial field's
    dissipation nu <omega^2>, computed here through the analysis module's own
    spectral derivatives, gives kappa_max eta = 1.5, kappa_max = sqrt(2) N / 3."""
    n = (32, 32, 32)
    mu0 = synth.mu0_for_resolution(n, k0=4.0, mach_t=0.3, seed=3)
    U = synth.initial_state(n, k0=4.0, mach_t=0.3, seed=3)
    rho, vel, p, T = analysis.primitives(U)
    om2 = float(analysis.enstrophy_field(analysis.gradients(vel)).mean())
    eta = (mu0 ** 3 / (mu0 * om2)) ** 0.25
    assert abs(math.sqrt(2.0) * 32 / 3.0 * eta - 1.5) < 1e-10


def test_synth_spectrum_shape():
    """The shell energy of the initial velocity follows k^4 exp(-2 (k/k0)^2)
    up to the sampling scatter of random amplitudes (shells 2..12 at 48^3)."""
    n = (48, 48, 48)
    U = synth.initial_state(n, k0=4.0, mach_t=0.3, seed=11)
    rho, vel, p, T = analysis.primitives(U)
    E = analysis.energy_spectrum(vel)
    k = np.arange(2, 13, dtype=float)
    ratio = E[2:13] / (k ** 4 * np.exp(-2.0 * (k / 4.0) ** 2))
    assert np.all(np.abs(ratio / np.median(ratio) - 1.0) < 0.35)
    assert E[20:].sum() < 1e-6 * E.sum()


def test_synth_history_levels():
    """history(): level l is U0 + (l + 1) eps dU, with a compressive dU (its
    velocity has a non-zero divergence) and a density perturbation."""
    n = (16, 12, 20)
    U0 = synth.initial_state(n, k0=3.0, mach_t=0.3, seed=2)
    h = synth.history(U0, 4, eps=1e-2, seed=5)
    d1, d2, d3 = h[1] - h[0], h[2] - h[1], h[3] - h[2]
    assert np.allclose(d1, d2, atol=1e-14) and np.allclose(d2, d3, atol=1e-14)
    assert np.allclose(h[0] - U0, d1, atol=1e-14)
    dvel = d1[1:4]
    div = sum(analysis.spectral_gradient(dvel[i])[i] for i in range(3))
    assert np.max(np.abs(div)) > 1e-4 and np.max(np.abs(d1[0])) > 1e-4
