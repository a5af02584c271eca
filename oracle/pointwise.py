"""Brute-force, one-point-at-a-time evaluation of the right-hand side.

TEST INFRASTRUCTURE ONLY (see ``oracle/ns.py``).

Each derivative is written out as an explicit list of (offset, time level,
weight) terms built from Table B (Appendix B): the standard stencil of the
configured order (4 or 6) repeated for l = 0 .. T_l-1, its points outside the
PE taken at level n-k-l and weighted by w_l(k) -- the same rows the paper
prints, read per point.  Under the other reading of what those weights
extrapolate (Config.extrapolate_state), a point outside the PE instead takes
the quantity of the extrapolated state sum_l w_l(k) U^{n-k-l} at that point,
once.  Mixed derivatives follow the three-step rule of
Sec. 2.1.  Pure Python loops, so it is used on tiny grids (as a brute-force
check of the vectorised oracle) and on a few hundred sampled points of
full-size grids (parity of the CUDA path).

The right-hand side is assembled from the definitions of Sec. 2 (total- or
internal-energy form, power-law or Sutherland viscosity): the
inviscid flux divergence, the viscous stress divergence
d sigma_ij/dx_j = mu (lap u_i + d theta/dx_i / 3)
                  + (d mu/dx_j)(du_i/dx_j + du_j/dx_i - 2/3 delta_ij theta),
the viscous work u_i d sigma_ij/dx_j + sigma_ij S_ij, the heat conduction
kappa lap T + (d kappa/dx_j)(dT/dx_j) and the forcing rho f_i, rho f_i u_i.
"""
import math

ENERGY_INTERNAL = 1     # the fifth variable is rho e (Eq. (ie)); 0: total energy E
VISC_SUTHERLAND = 1     # mu0 T^(3/2) (1 + S) / (T + S); 0: power law mu0 T^omega


class PointOracle:
    """RHS at single grid points.

    level(l) must return U^{n-l} as an array indexed [var, z, y, x] (it may be a
    numpy memmap or any object supporting that indexing).  delays[p][f] is the
    step's delay map; fhat the forcing coefficients (or None) with `modes`.
    """

    def __init__(self, cfg, level, delays, fhat=None, modes=None):
        self.cfg = cfg
        self.sc = cfg.scheme
        self.level = level
        self.delays = delays
        self.fhat = fhat
        self.modes = modes
        self._ucache = {}
        self._gcache = {}

    # ---- values at one point and one level ----------------------------
    def _wrap(self, pos):
        n = self.cfg.n
        return (pos[0] % n[0], pos[1] % n[1], pos[2] % n[2])

    def U(self, l, pos):
        """U at one point: l is a level index n-l, or ("x", k) for the state
        extrapolated to level n from the levels n-k-l with the weights w_l(k)."""
        pos = self._wrap(pos)
        key = (l, pos)
        if key not in self._ucache:
            if isinstance(l, tuple):
                k = l[1]
                w = self.sc.weights(k)
                self._ucache[key] = [sum(w[j] * self.U(k + j, pos)[v] for j in range(self.sc.T))
                                     for v in range(5)]
            else:
                lv = self.level(l)
                x, y, z = pos
                self._ucache[key] = [float(lv[v, z, y, x]) for v in range(5)]
        return self._ucache[key]

    def prim(self, l, pos):
        g = self.cfg.gamma
        rho, mx, my, mz, E = self.U(l, pos)
        u = (mx / rho, my / rho, mz / rho)
        if self.cfg.energy_form == ENERGY_INTERNAL:
            p = (g - 1.0) * E
        else:
            p = (g - 1.0) * (E - 0.5 * rho * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]))
        T = g * p / rho
        return rho, u, p, T

    def q(self, name, l, pos):
        rho, u, p, T = self.prim(l, pos)
        if name == "T":
            return T
        if name[0] == "u":
            return u[int(name[1])]
        d, e = int(name[1]), int(name[2])
        U = self.U(l, pos)
        if e == 0:
            return U[1 + d]
        if e == 4:
            return U[4] * u[d] if self.cfg.energy_form == ENERGY_INTERNAL else (U[4] + p) * u[d]
        i = e - 1
        return U[1 + i] * u[d] + (p if i == d else 0.0)

    # ---- geometry -------------------------------------------------------
    def pe_of(self, pos):
        pos = self._wrap(pos)
        nl = self.cfg.nloc
        px, py, pz = pos[0] // nl[0], pos[1] // nl[1], pos[2] // nl[2]
        return (pz * self.cfg.pes[1] + py) * self.cfg.pes[0] + px

    def local(self, pos, d):
        return self._wrap(pos)[d] % self.cfg.nloc[d]

    # ---- AT derivative as an explicit term list -------------------------
    def terms(self, pos, d, order):
        """[(offset, level, weight)] such that the derivative is
        sum weight * q(pos + offset e_d, level)."""
        cfg = self.cfg
        sc = self.sc
        if order == 1:
            stencil, denom = sc.d1, sc.d1_den * cfg.dx[d]
        else:
            stencil, denom = sc.d2, sc.d2_den * cfg.dx[d] ** 2
        if cfg.pes[d] == 1:
            return [(off, 0, c / denom) for off, c in stencil]
        nloc = cfg.nloc[d]
        li = self.local(pos, d)
        p = self.pe_of(pos)
        if li < sc.M:
            k = int(self.delays[p][2 * d])
        elif li >= nloc - sc.M:
            k = int(self.delays[p][2 * d + 1])
        else:
            k = 0
        if getattr(cfg, "extrapolate_state", False):
            return [(off, 0 if 0 <= li + off < nloc else ("x", k), c / denom)
                    for off, c in stencil]
        w = sc.weights(k)
        out = []
        for l in range(sc.T):
            for off, c in stencil:
                inside = 0 <= li + off < nloc
                out.append((off, 0 if inside else k + l, w[l] * c / denom))
        return out

    def deriv(self, name, pos, d, order):
        s = 0.0
        for off, lev, wt in self.terms(pos, d, order):
            p2 = list(pos)
            p2[d] += off
            s += wt * self.q(name, lev, tuple(p2))
        return s

    def grad(self, i, j, pos):
        """AT d u_i / d x_j at pos (cached)."""
        key = (i, j, self._wrap(pos))
        if key not in self._gcache:
            self._gcache[key] = self.deriv("u%d" % i, pos, j, 1)
        return self._gcache[key]

    # ---- mixed derivatives (Sec. 2.1) -----------------------------------
    def _central_fits(self, pos, d):
        if self.cfg.pes[d] == 1:
            return True
        li = self.local(pos, d)
        return self.sc.M <= li <= self.cfg.nloc[d] - 1 - self.sc.M

    def _pe_local_stencil(self, pos, d):
        if self.cfg.pes[d] == 1:
            return self.sc.d1
        return self.sc.one_sided(self.local(pos, d), self.cfg.nloc[d])

    def _apply_d1(self, stencil, gfun, pos, d):
        s = 0.0
        for off, c in stencil:
            p2 = list(pos)
            p2[d] += off
            s += c * gfun(tuple(p2))
        return s / (self.sc.d1_den * self.cfg.dx[d])

    def _plain_d1(self, name, lev, pos, b):
        """Central first derivative along b of quantity `name` at one level
        (an index, or ("x", k) for the extrapolated state), no PE faces."""
        s = 0.0
        for off, c in self.sc.d1:
            p2 = list(pos)
            p2[b] += off
            s += c * self.q(name, lev, tuple(p2))
        return s / (self.sc.d1_den * self.cfg.dx[b])

    def _ghost_grad(self, k, b, pos, kd):
        """The neighbour's d u_k / d x_b at an outside point, extrapolated to
        level n from the levels n-kd-l (or taken from the extrapolated state)."""
        name = "u%d" % k
        if getattr(self.cfg, "extrapolate_state", False):
            return self._plain_d1(name, ("x", kd), pos, b)
        w = self.sc.weights(kd)
        return sum(w[l] * self._plain_d1(name, kd + l, pos, b) for l in range(self.sc.T))

    def mixed(self, k, a, b, pos):
        """d/dx_a (d u_k / d x_b) at pos."""
        gb = lambda p: self.grad(k, b, p)
        ga = lambda p: self.grad(k, a, p)
        if getattr(self.cfg, "mixed_central", False):
            # central a-stencil at every point; beyond an a-face the
            # neighbour's extrapolated gradient
            if self.cfg.pes[a] == 1:
                return self._apply_d1(self.sc.d1, gb, pos, a)
            nloc = self.cfg.nloc[a]
            li = self.local(pos, a)
            p = self.pe_of(pos)
            kd = int(self.delays[p][2 * a]) if li < nloc // 2 else int(self.delays[p][2 * a + 1])
            s = 0.0
            for off, c in self.sc.d1:
                p2 = list(pos)
                p2[a] += off
                p2 = tuple(p2)
                s += c * (gb(p2) if 0 <= li + off < nloc else self._ghost_grad(k, b, p2, kd))
            return s / (self.sc.d1_den * self.cfg.dx[a])
        if self._central_fits(pos, a) and self._central_fits(pos, b):
            return self._apply_d1(self.sc.d1, gb, pos, a)
        return 0.5 * (self._apply_d1(self._pe_local_stencil(pos, a), gb, pos, a)
                      + self._apply_d1(self._pe_local_stencil(pos, b), ga, pos, b))

    # ---- forcing ---------------------------------------------------------
    def force(self, pos):
        if self.fhat is None:
            return (0.0, 0.0, 0.0)
        cfg = self.cfg
        x = [self._wrap(pos)[d] * cfg.dx[d] for d in range(3)]
        f = [0.0, 0.0, 0.0]
        for m, (kx, ky, kz) in enumerate(self.modes):
            ph = kx * x[0] + ky * x[1] + kz * x[2]
            cph, sph = math.cos(ph), math.sin(ph)
            for c in range(3):
                fh = complex(self.fhat[m][c])
                f[c] += 2.0 * (fh.real * cph - fh.imag * sph)
        return tuple(f)

    # ---- the right-hand side at one point --------------------------------
    def rhs(self, pos):
        cfg = self.cfg
        g = cfg.gamma
        R = [0.0] * 5
        for d in range(3):
            for e in range(5):
                R[e] -= self.deriv("F%d%d" % (d, e), pos, d, 1)
        rho, u, p, T = self.prim(0, pos)
        A = [[self.grad(i, j, pos) for j in range(3)] for i in range(3)]
        dT = [self.deriv("T", pos, j, 1) for j in range(3)]
        d2u = [[self.deriv("u%d" % i, pos, j, 2) for j in range(3)] for i in range(3)]
        lapT = sum(self.deriv("T", pos, j, 2) for j in range(3))
        theta = A[0][0] + A[1][1] + A[2][2]
        dtheta = []
        for i in range(3):
            s = d2u[i][i]
            for k in range(3):
                if k != i:
                    s += self.mixed(k, i, k, pos)
            dtheta.append(s)
        if cfg.visc_law == VISC_SUTHERLAND:
            S = cfg.suth_s
            mu = cfg.mu0 * T * math.sqrt(T) * (1.0 + S) / (T + S)
            dmu_dT = mu * (1.5 / T - 1.0 / (T + S))
        else:
            mu = cfg.mu0 * T ** cfg.visc_exp
            dmu_dT = cfg.visc_exp * mu / T
        dmu = [dmu_dT * dT[j] for j in range(3)]
        cp = 1.0 / (g - 1.0)
        kappa = mu * cp / cfg.prandtl
        f = self.force(pos)
        work = 0.0
        for i in range(3):
            V = mu * (sum(d2u[i]) + dtheta[i] / 3.0)
            for j in range(3):
                V += dmu[j] * (A[i][j] + A[j][i] - (2.0 / 3.0 if i == j else 0.0) * theta)
            R[1 + i] += V + rho * f[i]
            work += u[i] * V
        sigS = 0.0
        for i in range(3):
            for j in range(3):
                sig = mu * (A[i][j] + A[j][i] - (2.0 / 3.0 if i == j else 0.0) * theta)
                sigS += sig * 0.5 * (A[i][j] + A[j][i])
        heat = kappa * lapT + sum(dmu[j] * cp / cfg.prandtl * dT[j] for j in range(3))
        if cfg.energy_form == ENERGY_INTERNAL:
            R[4] += -p * theta + sigS + heat
        else:
            R[4] += work + sigS + heat + sum(rho * f[i] * u[i] for i in range(3))
        return R
