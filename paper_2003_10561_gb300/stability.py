"""Stability limits of AT schemes under a fixed worst-case delay (Sec. 3.2
and Appendix A), computed on the host.

Model problem: the 1D diffusion equation du/dt = alpha d2u/dx2 with one grid
point per PE (P = N), so every stencil neighbour lies across a PE face and
reads delayed levels.  With a Fourier mode u_i^n = v^n exp(I i phi) the
scheme becomes a linear recurrence v^{n+1} = sum_m c_m(phi) v^{n-m}; its
Z-transform is the polynomial z^(K+1) - sum_m c_m z^(K-m), and the scheme is
stable when every root lies in the unit disc for every phi (the root z = 1 at
phi = 0 is the steady state).  The largest stable diffusive CFL
r_d = alpha dt / dx^2 is found by bisection; f(L) = r_d,max(0) / r_d,max(L)
is the factor by which a delay L shrinks it (Eq. (rdml)).

Schemes:
* order 2 with forward Euler (Eq. (dis_at)): the neighbours are taken as
  (k+1) u^{n-k} - k u^{n-k-1};
* order 4 with AB2 (the scheme of the turbulence runs): the neighbours of
  the 4th-order central D2 are taken with the Table B weights of levels
  n-k, n-k-1, n-k-2.
Delays act on both faces (the paper's worst case) or on one face only.

The companion-matrix form of Sec. 3.2 (V^{n+1} = A V^n for a periodic line of
N points) is built for the order-2 scheme as an independent check: its
spectral radius equals the largest root modulus over the N discrete phases.

In the printed Z-transform (Appendix A) the neighbour factor reads
e^{-I phi} - e^{I phi} and the last term carries the wrong sign; the
polynomial is derived here directly from Eq. (vn2):
z^{L+2} - (1 - 2 r_d) z^{L+1} - 2 r_d cos(phi) ((L+1) z - L) = 0.
"""
import numpy as np


def _at_weights(k, order):
    if order == 2:
        return [k + 1.0, -float(k)]
    return [(k * k + 3.0 * k + 2.0) / 2.0, -(k * k + 2.0 * k), (k * k + k) / 2.0]


def recurrence(L, rd, phi, order=2, one_sided=False):
    """Coefficients c_m (m = 0, 1, ...) of v^{n+1} = sum_m c_m v^{n-m}."""
    w = _at_weights(L, order)
    K = L + len(w) + (1 if order == 4 else 0)      # deepest level read (AB2 adds one)
    c = np.zeros(K + 1, dtype=complex)
    if order == 2:
        left, right = rd * np.exp(-1j * phi), rd * np.exp(1j * phi)
        c[0] += 1.0 - 2.0 * rd
        for side, coef in ((0, left), (1, right)):
            if one_sided and side == 1:
                c[0] += coef
            else:
                for l, wl in enumerate(w):
                    c[L + l] += coef * wl
        return c
    # order 4, AB2: S^n = rd/12 [-30 v^n + neighbours], v^{n+1} = v^n + 3/2 S^n - 1/2 S^{n-1}
    s = np.zeros(K + 1, dtype=complex)
    left = rd / 12.0 * (16.0 * np.exp(-1j * phi) - np.exp(-2j * phi))
    right = rd / 12.0 * (16.0 * np.exp(1j * phi) - np.exp(2j * phi))
    s[0] += -30.0 * rd / 12.0
    for side, coef in ((0, left), (1, right)):
        if one_sided and side == 1:
            s[0] += coef
        else:
            for l, wl in enumerate(w):
                s[L + l] += coef * wl
    c[0] += 1.0
    c += 1.5 * s
    c[1:] += -0.5 * s[:-1]
    return c


def roots(L, rd, phi, order=2, one_sided=False):
    """Roots in z of the Z-transform of the recurrence."""
    c = recurrence(L, rd, phi, order, one_sided)
    return np.roots(np.concatenate([[1.0], -c]))


def spectral_radius(L, rd, order=2, one_sided=False, nphi=181):
    """max over phi in [0, pi] of the largest root modulus."""
    return max(float(np.max(np.abs(roots(L, rd, ph, order, one_sided)))) for ph in np.linspace(0.0, np.pi, nphi))


def rd_max(L, order=2, one_sided=False, tol=1e-6, slack=1e-9, nphi=181):
    """Largest diffusive CFL with every root in the unit disc (bisection)."""
    lo, hi = 0.0, 1.0
    while hi - lo > tol:
        mid = 0.5 * (lo + hi)
        if spectral_radius(L, mid, order, one_sided, nphi) <= 1.0 + slack:
            lo = mid
        else:
            hi = mid
    return lo


def fit_f(Ls, rds, deg):
    """Polynomial fit of f(L) = r_d,max(0) / r_d,max(L) (coefficients, highest first)."""
    f = rds[0] / np.asarray(rds)
    return np.polyfit(np.asarray(Ls, dtype=float), f, deg)


def companion_matrix(N, L, rd):
    """Sec. 3.2 evolution matrix of the order-2 forward-Euler AT scheme on a
    periodic line of N one-point PEs with delay L on both faces:
    V^{n+1} = A V^n, V^n = [U^n, U^{n-1}, ..., U^{n-L-1}]."""
    blocks = L + 2
    A = np.zeros((blocks * N, blocks * N))
    idx = np.arange(N)
    A[idx, idx] += 1.0 - 2.0 * rd
    for l, wl in enumerate(_at_weights(L, 2)):
        col = (L + l) * N
        A[idx, col + (idx - 1) % N] += rd * wl
        A[idx, col + (idx + 1) % N] += rd * wl
    for b in range(1, blocks):
        A[b * N + idx, (b - 1) * N + idx] = 1.0
    return A


def ns_cfl_limit(make_solver, state, L, steps=400, lo=0.05, hi=2.0, tol=0.01, growth=1.5):
    """Largest convective CFL at which the Navier-Stokes solver stays stable
    for `steps` AB2 steps with the fixed delay L on every face (Sec. 3.2:
    bisection on the CFL with the worst-case delay).

    make_solver(cfl) returns a Solver (at_dns.Solver) whose dt comes from that
    CFL; a run is unstable when the library reports a non-finite or
    non-positive state, or when the kinetic energy of the decaying flow grows
    by the factor `growth`."""
    from . import at_dns

    def stable(cfl):
        s = make_solver(cfl)
        try:
            s.set_state(state)
            k0 = s.stats()["tke"]
            s.step(steps, "fixed" if L > 0 else "sync")
            ok = s.stats()["tke"] <= growth * k0
        except at_dns.AtDnsError as e:
            if e.code != at_dns.AT_DNS_E_UNSTABLE:
                raise
            ok = False
        finally:
            s.close()
        return ok

    if not stable(lo):
        return 0.0
    while hi - lo > tol:
        mid = 0.5 * (lo + hi)
        if stable(mid):
            lo = mid
        else:
            hi = mid
    return lo
