"""Manufactured smooth fields and the exact right-hand side of the compressible
Navier-Stokes equations, derived symbolically with sympy from the conservation
laws in divergence form (Sec. 2, Eqs. (cont), (mome) and the total-energy
equation d E/dt + d((E+p)u_j)/dx_j = d(u_i sigma_ij)/dx_j + d(k dT/dx_j)/dx_j).

Nothing here is shared with the oracle's discretisation: the derivatives are
sympy's, the viscous terms stay in divergence form, and the result is the
exact time derivative of the conserved variables.
"""
import functools

import numpy as np
import sympy as sp

x, y, z, t = sp.symbols("x y z t", real=True)


def fields(mixed=False):
    """Smooth periodic rho, u, v, w, T (functions of x, y, z, t).

    In the default set each d u_k/d x_k depends on x_k alone and not on t, so
    the mixed terms d/dx_i (d u_k/dx_k), i != k, of the viscous stress vanish
    identically.  mixed=True multiplies each of those parts by a travelling
    wave in another direction, so that every d u_k/d x_k depends on two
    coordinates and on t, and d/dy (du/dx), d/dz (dv/dy) and d/dx (dw/dz) --
    a mixed term with each direction outermost -- are nonzero."""
    rho = 1 + sp.Rational(1, 10) * sp.sin(x + sp.Rational(3, 10) * t) * sp.cos(y) \
        + sp.Rational(1, 20) * sp.sin(z - sp.Rational(1, 5) * t)
    if mixed:
        fu = sp.sin(y + sp.Rational(1, 5) * t)
        fv = sp.cos(z - sp.Rational(3, 10) * t)
        fw = sp.sin(x + sp.Rational(1, 4) * t)
    else:
        fu = fv = fw = 1
    u = sp.Rational(1, 5) * sp.sin(y) * sp.cos(z + sp.Rational(1, 10) * t) + sp.Rational(1, 10) * sp.cos(x) * fu
    v = sp.Rational(3, 20) * sp.sin(z) * sp.cos(x - sp.Rational(1, 5) * t) + sp.Rational(1, 20) * sp.sin(y) * fv
    w = sp.Rational(1, 10) * sp.sin(x) * sp.sin(y + sp.Rational(3, 10) * t) + sp.Rational(2, 25) * sp.cos(z) * fw
    T = 1 + sp.Rational(1, 10) * sp.cos(x - y) * sp.sin(z + sp.Rational(1, 5) * t)
    return rho, (u, v, w), T


@functools.lru_cache(maxsize=None)
def exact(gamma, prandtl, mu0, omega, internal=False, sutherland=None, mixed=False):
    """Return (conserved(X, Y, Z, tt), rhs(X, Y, Z, tt)) numpy callables.

    internal: the fifth variable is rho e with the paper's Eq. (ie),
    d(rho e)/dt + d(rho e u_j)/dx_j = -p du_j/dx_j + d(k dT/dx_j)/dx_j
    + sigma_ij S_ij; else total energy.  sutherland = S: Sutherland's law
    mu0 T^(3/2) (1 + S) / (T + S) instead of the power law.  mixed: the
    field set whose mixed viscous terms are nonzero (fields(mixed=True))."""
    g = sp.nsimplify(gamma)
    rho, vel, T = fields(mixed)
    X = (x, y, z)
    p = rho * T / g
    E = p / (g - 1) + rho * (vel[0] ** 2 + vel[1] ** 2 + vel[2] ** 2) / 2
    if sutherland is None:
        mu = sp.nsimplify(mu0) * T ** sp.nsimplify(omega)
    else:
        S = sp.nsimplify(sutherland)
        mu = sp.nsimplify(mu0) * T ** sp.Rational(3, 2) * (1 + S) / (T + S)
    kap = mu / (g - 1) / sp.nsimplify(prandtl)
    dudx = [[sp.diff(vel[i], X[j]) for j in range(3)] for i in range(3)]
    theta = dudx[0][0] + dudx[1][1] + dudx[2][2]
    sigma = [[mu * (dudx[i][j] + dudx[j][i] - (sp.Rational(2, 3) * theta if i == j else 0))
              for j in range(3)] for i in range(3)]
    R = [0] * 5
    R[0] = -sum(sp.diff(rho * vel[j], X[j]) for j in range(3))
    for i in range(3):
        R[1 + i] = sum(-sp.diff(rho * vel[i] * vel[j] + (p if i == j else 0), X[j])
                       + sp.diff(sigma[i][j], X[j]) for j in range(3))
    if internal:
        rhoe = p / (g - 1)
        R[4] = sum(-sp.diff(rhoe * vel[j], X[j]) - p * dudx[j][j]
                   + sp.diff(kap * sp.diff(T, X[j]), X[j]) for j in range(3)) \
            + sum(sigma[i][j] * (dudx[i][j] + dudx[j][i]) / 2 for i in range(3) for j in range(3))
        last = rhoe
    else:
        R[4] = sum(-sp.diff((E + p) * vel[j], X[j])
                   + sp.diff(sum(vel[i] * sigma[i][j] for i in range(3)), X[j])
                   + sp.diff(kap * sp.diff(T, X[j]), X[j]) for j in range(3))
        last = E
    cons = [rho, rho * vel[0], rho * vel[1], rho * vel[2], last]
    fc = sp.lambdify((x, y, z, t), cons, "numpy")
    fr = sp.lambdify((x, y, z, t), R, "numpy")
    return fc, fr


def grid(n):
    """[z, y, x] coordinate arrays of the (2 pi)^3 grid."""
    ax = [np.arange(m) * 2 * np.pi / m for m in n]
    Z, Y, X = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    return X, Y, Z


def evaluate(f, n, tt):
    X, Y, Z = grid(n)
    out = f(X, Y, Z, tt)
    return np.stack([np.broadcast_to(np.asarray(o, dtype=np.float64), X.shape) for o in out])
