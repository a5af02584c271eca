"""Host analysis of state snapshots (numpy): the spectra, PDFs and slices
the paper uses to compare synchronous and asynchronous runs (Sec. 4.1).

Input is a state as returned by ``Solver.get_state()`` -- FP64
[5][nz][ny][nx] with the fifth variable E (total-energy form) or rho e
(internal-energy form) -- on the periodic (2 pi)^3 box.  Derivatives here are
spectral (exact for the grid's band-limited interpolant), so the analysis is
independent of the finite differences it is used to check.

Definitions (nondimensional, rho_0 = T_0 = c_0 = 1):

* energy spectrum E(kappa) = sum over the shell kappa - 1/2 <= |k| <
  kappa + 1/2 of |u_hat_i(k)|^2 / 2, u_hat the discrete Fourier coefficients
  of the velocity divided by N^3, so that sum_kappa E = <u_i u_i>/2
  (Eq. (ener));
* pressure spectrum E_p(kappa): the same shell sum of |p_hat(k)|^2 over
  k != 0, so that sum_kappa E_p = <p'p'>; it is formed from the kinematic
  pressure p / <rho>;
* mean dissipation per unit mass <eps> = <sigma_ij S_ij> / <rho>, kinematic
  viscosity nu = <mu> / <rho>, Kolmogorov scale eta = (nu^3/<eps>)^(1/4);
* compensated spectra E / (<eps>^(2/3) kappa^(-5/3)) (Eq. (ener1)) and
  E_p <eps>^(-4/3) kappa^(7/3), plotted against kappa eta;
* enstrophy Omega = <omega_i omega_i>, skewness and flatness of the
  longitudinal gradients (Sec. 4.1.3);
* PDFs of eps / <eps> and Omega / <Omega> (normalised histograms), and a
  z-slice of omega_i omega_i / <omega_i omega_i> (Sec. 4.1.4).
"""
import math

import numpy as np

ENERGY_TOTAL, ENERGY_INTERNAL = 0, 1


def wavenumbers(n):
    """Integer wavenumber arrays kx, ky, kz broadcastable over a [z, y, x]
    field, in numpy's FFT order (Nyquist as -n/2)."""
    k = [np.fft.fftfreq(m, 1.0 / m) for m in n]
    return (k[0].reshape(1, 1, -1), k[1].reshape(1, -1, 1), k[2].reshape(-1, 1, 1))


def primitives(U, gamma=1.4, energy_form=ENERGY_TOTAL):
    """rho, velocity (3 arrays), p, T of a state."""
    rho = U[0]
    vel = [U[1] / rho, U[2] / rho, U[3] / rho]
    if energy_form == ENERGY_INTERNAL:
        p = (gamma - 1.0) * U[4]
    else:
        p = (gamma - 1.0) * (U[4] - 0.5 * rho * (vel[0] ** 2 + vel[1] ** 2 + vel[2] ** 2))
    return rho, vel, p, gamma * p / rho


def spectral_gradient(f):
    """[df/dx, df/dy, df/dz] of a periodic field on the (2 pi)^3 box; the
    Nyquist modes are dropped (their derivative is not defined)."""
    n = (f.shape[2], f.shape[1], f.shape[0])
    fh = np.fft.fftn(f)
    out = []
    for d, k in enumerate(wavenumbers(n)):
        kk = k.copy()
        if n[d] % 2 == 0:
            kk[kk == -n[d] // 2] = 0.0
        out.append(np.real(np.fft.ifftn(1j * kk * fh)))
    return out


def shell_sum(power, n):
    """Sum of a [z, y, x] array of modal powers over the shells
    kappa - 1/2 <= |k| < kappa + 1/2, kappa = 0, 1, ..."""
    kx, ky, kz = wavenumbers(n)
    kmag = np.sqrt(kx * kx + ky * ky + kz * kz)
    shell = np.floor(kmag + 0.5).astype(np.int64)
    return np.bincount(shell.ravel(), weights=power.ravel())


def energy_spectrum(vel):
    """E(kappa) of a velocity field (list of three [z, y, x] arrays)."""
    n = (vel[0].shape[2], vel[0].shape[1], vel[0].shape[0])
    N3 = float(vel[0].size)
    power = sum(np.abs(np.fft.fftn(u) / N3) ** 2 for u in vel) * 0.5
    return shell_sum(power, n)


def pressure_spectrum(p):
    """E_p(kappa) of a (kinematic) pressure field, mean removed."""
    n = (p.shape[2], p.shape[1], p.shape[0])
    ph = np.fft.fftn(p - p.mean()) / float(p.size)
    return shell_sum(np.abs(ph) ** 2, n)


def gradients(vel):
    """A[i][j] = d u_i / d x_j (spectral)."""
    return [spectral_gradient(u) for u in vel]


def dissipation_field(A, mu):
    """sigma_ij S_ij with sigma = mu (A + A^T - 2/3 theta I), S = (A + A^T)/2."""
    theta = A[0][0] + A[1][1] + A[2][2]
    out = np.zeros_like(theta)
    for i in range(3):
        for j in range(3):
            s = 0.5 * (A[i][j] + A[j][i])
            out += mu * (A[i][j] + A[j][i] - (2.0 / 3.0 if i == j else 0.0) * theta) * s
    return out


def enstrophy_field(A):
    o = [A[2][1] - A[1][2], A[0][2] - A[2][0], A[1][0] - A[0][1]]
    return o[0] ** 2 + o[1] ** 2 + o[2] ** 2


def normalized_pdf(x, bins=64, log=True):
    """Histogram density of x / <x> (log-spaced bins for positive fields);
    returns (bin centres, density) with sum(density * widths) = 1."""
    y = np.asarray(x, dtype=np.float64).ravel()
    y = y / y.mean()
    if log:
        y = y[y > 0]
        edges = np.logspace(np.log10(y.min()), np.log10(y.max()) * (1 + 1e-12), bins + 1)
    else:
        edges = np.linspace(y.min(), y.max() * (1 + 1e-12) if y.max() > 0 else y.max() + 1e-12, bins + 1)
    dens, edges = np.histogram(y, bins=edges, density=True)
    return 0.5 * (edges[1:] + edges[:-1]), dens


def analyze(U, mu0=0.01, visc_exp=0.76, gamma=1.4, energy_form=ENERGY_TOTAL, visc_law=0, suth_s=0.368,
            bins=64):
    """All the Sec. 4.1 diagnostics of one snapshot, as a dict."""
    rho, vel, p, T = primitives(U, gamma, energy_form)
    if visc_law == 1:
        mu = mu0 * T ** 1.5 * (1.0 + suth_s) / (T + suth_s)
    else:
        mu = mu0 * T ** visc_exp
    A = gradients(vel)
    eps_f = dissipation_field(A, mu)
    ens_f = enstrophy_field(A)
    rho_m = float(rho.mean())
    eps = float(eps_f.mean()) / rho_m
    nu = float(mu.mean()) / rho_m
    eta = (nu ** 3 / eps) ** 0.25 if eps > 0 else float("inf")
    E = energy_spectrum(vel)
    Ep = pressure_spectrum(p / rho_m)
    kap = np.arange(len(E), dtype=np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        comp = np.where(kap > 0, E / (eps ** (2.0 / 3.0) * kap ** (-5.0 / 3.0)), 0.0)
        comp_p = np.where(kap > 0, Ep * eps ** (-4.0 / 3.0) * kap ** (7.0 / 3.0), 0.0)
    m2 = np.mean([np.mean(A[i][i] ** 2) for i in range(3)])
    m3 = np.mean([np.mean(A[i][i] ** 3) for i in range(3)])
    m4 = np.mean([np.mean(A[i][i] ** 4) for i in range(3)])
    u2 = float(np.mean(vel[0] ** 2 + vel[1] ** 2 + vel[2] ** 2))
    urms = math.sqrt(u2 / 3.0)
    lam = math.sqrt(15.0 * nu * urms ** 2 / eps) if eps > 0 else float("inf")   # Taylor microscale
    n = U.shape[1:]
    kmax = math.sqrt(2.0) * min(n) / 3.0
    mid = U.shape[1] // 2
    return {
        "kappa": kap, "E": E, "Ep": Ep, "kappa_eta": kap * eta, "E_compensated": comp, "Ep_compensated": comp_p,
        "eps": eps, "nu": nu, "eta": eta, "kmax_eta": kmax * eta, "urms": urms, "taylor": lam,
        "re_lambda": urms * lam / nu if nu > 0 else float("inf"),
        "enstrophy": float(ens_f.mean()), "skewness": m3 / m2 ** 1.5, "flatness": m4 / m2 ** 2,
        "pdf_eps": normalized_pdf(eps_f, bins), "pdf_enstrophy": normalized_pdf(ens_f, bins),
        "pdf_gradient": normalized_pdf(A[0][0] / math.sqrt(np.mean(A[0][0] ** 2)), bins, log=False),
        "enstrophy_slice": ens_f[mid] / ens_f.mean(),
    }


def forced_stationary_state(solver, state, block=200, max_blocks=50, tol=0.02, mode="sync"):
    """Advance a forced solver (at_dns.Solver with forcing on) from `state`
    until the kinetic energy is statistically stationary: the mean of K over
    the last block of steps differs from the previous block's by less than
    `tol` (relative).  Stands in for the paper's forced stationary fields
    (Sec. 4.2), which are not available.  Returns (state, K history per block)."""
    solver.set_state(state)
    history = []
    prev = None
    for _ in range(max_blocks):
        ks = []
        for _ in range(max(1, block // 10)):
            solver.step(10, mode)
            ks.append(solver.stats()["tke"])
        mean = float(np.mean(ks))
        history.append(mean)
        if prev is not None and abs(mean - prev) <= tol * abs(prev):
            break
        prev = mean
    return solver.get_state(), history
