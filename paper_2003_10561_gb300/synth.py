"""Seeded synthetic inputs shaped like the paper's runs (Sec. 4, Table 3).

This module only builds inputs.  It holds none of the solver's arithmetic and
imports neither the CUDA library nor the oracle, so tests, the benchmark and the
oracle can all take their inputs from it.

Initial field: periodic (2 pi)^3 box, uniform density and temperature
(rho = 1, T = 1 in units where c_0 = 1, so p = 1/gamma), and a random-phase
solenoidal velocity with energy spectrum E(k) ~ k^4 exp(-2 (k/k0)^2), scaled so
that the turbulent Mach number <u_i u_i>^{1/2} / c_0 equals ``mach_t``
(M_t ~ 0.3 in the paper, Sec. 4).  Conserved variables are
(rho, rho u, rho v, rho w, E) with E = p/(gamma-1) + rho |u|^2 / 2.  The paper
starts from forced stationary fields that are not available; this spectrum is
the stand-in.

Arrays are float64, shape (5, nz, ny, nx), x fastest (C order).
"""
import math

import numpy as np


def _wavenumbers(n):
    nx, ny, nz = n
    kx = np.fft.fftfreq(nx, 1.0 / nx)
    ky = np.fft.fftfreq(ny, 1.0 / ny)
    kz = np.fft.fftfreq(nz, 1.0 / nz)
    KZ, KY, KX = np.meshgrid(kz, ky, kx, indexing="ij")
    return KX, KY, KZ


def solenoidal_velocity(n, k0=4.0, mach_t=0.3, seed=0):
    """Random solenoidal velocity (u, v, w), each (nz, ny, nx), zero mean."""
    rng = np.random.Generator(np.random.PCG64(seed))
    KX, KY, KZ = _wavenumbers(n)
    k2 = KX ** 2 + KY ** 2 + KZ ** 2
    kmag = np.sqrt(k2)
    # shell-averaged |u_hat(k)|^2 ~ E(k) / k^2  ->  amplitude ~ k exp(-(k/k0)^2)
    amp = kmag * np.exp(-(kmag / k0) ** 2)
    amp[k2 == 0] = 0.0
    shape = (3,) + k2.shape
    noise = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    uh = noise * amp
    # remove the component along k (projection onto divergence-free fields)
    kk = np.stack([KX, KY, KZ])
    k2s = np.where(k2 == 0, 1.0, k2)
    kdotu = (kk * uh).sum(axis=0) / k2s
    uh = uh - kk * kdotu
    # zero the Nyquist planes so the real part stays exactly solenoidal
    for d, K in enumerate((KX, KY, KZ)):
        nyq = n[d] // 2 if n[d] % 2 == 0 else None
        if nyq is not None:
            uh[:, np.abs(K) == nyq] = 0.0
    u = np.real(np.fft.ifftn(uh, axes=(1, 2, 3)))
    u -= u.mean(axis=(1, 2, 3), keepdims=True)
    scale = mach_t / math.sqrt(float(np.mean((u ** 2).sum(axis=0))))
    return u * scale


def initial_state(n, k0=4.0, mach_t=0.3, seed=0, gamma=1.4):
    """Conserved variables (5, nz, ny, nx) of the decaying-turbulence start."""
    vel = solenoidal_velocity(n, k0, mach_t, seed)
    rho = np.ones(vel.shape[1:])
    p = np.full(vel.shape[1:], 1.0 / gamma)
    U = np.empty((5,) + vel.shape[1:])
    U[0] = rho
    U[1:4] = rho * vel
    U[4] = p / (gamma - 1.0) + 0.5 * rho * (vel ** 2).sum(axis=0)
    return U


def mu0_for_resolution(n, k0=4.0, mach_t=0.3, seed=0, kmax_eta=1.5):
    """Viscosity that gives kappa_max eta = kmax_eta at t = 0 (Sec. 4):
    kappa_max = sqrt(2) N / 3, eta = (nu^3/eps)^(1/4), eps = nu <omega^2>
    from the spectral vorticity of the initial field, rho = 1."""
    vel = solenoidal_velocity(n, k0, mach_t, seed)
    KX, KY, KZ = _wavenumbers(n)
    uh = np.fft.fftn(vel, axes=(1, 2, 3)) / float(np.prod(n))
    k2 = KX ** 2 + KY ** 2 + KZ ** 2
    # <omega_i omega_i> = <|k|^2 |u_hat|^2> for a solenoidal field (Parseval)
    om2 = float(np.sum(k2 * (np.abs(uh) ** 2).sum(axis=0)))
    kmax = math.sqrt(2.0) * n[0] / 3.0
    eta = kmax_eta / kmax
    return eta * eta * math.sqrt(om2)


def history(U0, n_levels, eps=1e-3, seed=1):
    """A smooth synthetic past [U^n, U^{n-1}, ...]: level l is U0 plus (l + 1)
    times a small seeded smooth perturbation with a compressive part (so that
    the delayed levels differ and no right-hand side component is degenerate,
    e.g. a vanishing mass flux divergence of an exactly solenoidal field)."""
    n = (U0.shape[3], U0.shape[2], U0.shape[1])
    dvel = solenoidal_velocity(n, 3.0, 1.0, seed)
    rng = np.random.Generator(np.random.PCG64(seed + 7))
    phase = rng.uniform(0, 2 * math.pi, 3)
    z, y, x = np.meshgrid(*(np.arange(m) * 2 * math.pi / m for m in (n[2], n[1], n[0])), indexing="ij")
    drho = np.sin(x + phase[0]) * np.cos(y + phase[1]) * np.sin(2 * z + phase[2])
    dU = np.empty_like(U0)
    # irrotational (compressive) velocity part: gradient of a smooth potential
    a, b, c = phase
    grad_phi = np.stack([np.cos(x + a) * np.sin(y + b) * np.cos(z + c),
                         np.sin(x + a) * np.cos(y + b) * np.cos(z + c),
                         -np.sin(x + a) * np.sin(y + b) * np.sin(z + c)])
    dU[0] = 0.05 * drho
    dU[1:4] = dvel * 0.1 + 0.2 * grad_phi
    dU[4] = 0.1 * drho
    return [U0 + ((l + 1) * eps) * dU for l in range(n_levels)]
