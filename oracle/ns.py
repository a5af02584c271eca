"""FP64 CPU oracle for one time step of the compressible Navier-Stokes equations
with Asynchrony-Tolerant (AT) stencils at the faces of virtual PEs.

TEST INFRASTRUCTURE ONLY.  Plain, slow, vectorised numpy written from the paper
(Kumari & Donzis, arXiv 2003.10561).  It is imported only by ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``; the
product path never imports it and shares no code with it.

Paper passages followed, in the order of one step:

* delay map: control parameters c_r and L (Sec. 3.1), random delays of the
  Synchronization-Avoiding Algorithm (Algorithm 1, Sec. 3.1.1), periodic
  delays of the Communication-Avoiding Algorithm (Algorithm 2, Sec. 3.1.2),
  synchronous start-up over the first L + T_l steps (Algorithms 1 and 2);
* AT derivatives at PE faces: Eq. (at) and the 4th-order rows of Table B
  (Appendix B), standard 4th-order stencils at internal points (Sec. 2.1);
  optionally the 6th-order rows of Table B (T_l = 4) with standard 6th-order
  stencils inside (the sixth-order comparison of Sec. 4.1.2);
* mixed derivatives in three steps at boundary points (Sec. 2.1);
* right-hand side of Eqs. (cont), (mome) and the energy equation with the
  stress / strain definitions of Sec. 2 (total energy form, see below);
* large-scale solenoidal forcing in a shell |kappa| <= kappa_f (Sec. 4.2);
* second-order Adams-Bashforth, Eq. (time_ab) with T = 2 (Sec. 2.2); or, for
  synchronous runs only, a low-storage three-stage Runge-Kutta scheme
  (Williamson, J. Comput. Phys. 35, 1980: dU = A_s dU + dt R, U = U + B_s dU,
  A = (0, -5/9, -153/128), B = (1/3, 15/16, 8/15)) -- the paper discusses
  RK and keeps AB2 for AT because each RK stage would need a synchronisation.

Readings where the paper is silent:

* Non-dimensionalisation rho_0 = T_0 = c_0 = 1, so R = 1/gamma,
  p = rho T / gamma, c^2 = T, c_p = 1/(gamma-1).
* Energy variable: total energy E = rho e + rho |u|^2 / 2 in divergence form
  (default); the viscous work and conduction terms are expanded into first,
  second and mixed derivatives (the paper's derivative machinery).  Or the
  paper's own internal-energy form, Eq. (ie): the fifth variable is rho e and
  its right-hand side is -d(rho e u_j)/dx_j - p theta + sigma_ij S_ij
  + d(k dT/dx_j)/dx_j.
* Viscosity: power law mu = mu0 T^omega (default), or Sutherland's law
  mu = mu0 T^(3/2) (1 + S) / (T + S) with S the Sutherland temperature over
  the reference temperature (the paper names the law without constants;
  S = 110.4 K / 300 K = 0.368 is taken).
* Only stencil points outside the PE read delayed levels; the two sides of a
  shared face have independent delays; a direction with one PE has no faces.
* Quantity extrapolated by the AT weights: the differentiated quantity
  (flux, velocity component, temperature) evaluated at each delayed level.
  Config.extrapolate_state takes the other reading: the state U is
  extrapolated to level n first and the quantity evaluated once from it.
* Mixed derivatives at PE faces: the three-step rule with one-sided stencils
  (Sec. 2.1).  Config.mixed_central takes the other reading: the central
  stencil everywhere, over the neighbour's gradient extrapolated with the
  Table B weights beyond a face, so that zero delays give the single-PE
  scheme.
* AB2 start: the first step after a state is set is a forward-Euler step.
* Random delays: iid uniform on {0..L} from Philox4x32-10; periodic delays
  k = (n - n0) mod c_r; n0 = L + T_l synchronous start-up steps.
* Forcing: an Ornstein-Uhlenbeck process per Fourier mode (the Eswaran-Pope
  scheme cited by the paper is not reproduced in it).
"""
from dataclasses import dataclass, field
import math

import numpy as np

from .philox import philox4x32_10, split_seed
from .stencils import Scheme

SYNC, PERIODIC, RANDOM, FIXED, ORDERED = 0, 1, 2, 3, 4
ENERGY_TOTAL, ENERGY_INTERNAL = 0, 1
VISC_POWER, VISC_SUTHERLAND = 0, 1
AB2, RK3 = 0, 1
RK3_A = (0.0, -5.0 / 9.0, -153.0 / 128.0)
RK3_B = (1.0 / 3.0, 15.0 / 16.0, 8.0 / 15.0)
DELAY_STREAM_TAG = 0x4154      # 4th Philox counter word of the delay stream
FORCING_STREAM_TAG = 0x464F    # 4th Philox counter word of the forcing stream


@dataclass
class Config:
    n: tuple = (32, 32, 32)          # grid points (nx, ny, nz)
    pes: tuple = (1, 1, 1)           # virtual PEs (Px, Py, Pz)
    gamma: float = 1.4
    prandtl: float = 0.7
    mu0: float = 0.02
    visc_exp: float = 0.76
    dt: float = 1e-3
    max_delay: int = 2               # L
    comm_period: int = 3             # c_r (periodic mode)
    seed: int = 0                    # delay stream seed
    forcing: bool = False
    kf: float = 2.0
    f_amp: float = 0.0
    f_tcorr: float = 1.0
    f_seed: int = 0
    order: int = 4                   # spatial order: 4 (T_l = 3) or 6 (T_l = 4)
    energy_form: int = ENERGY_TOTAL  # fifth variable: E (total) or rho e (Eq. (ie))
    visc_law: int = VISC_POWER       # mu0 T^omega, or Sutherland with S = suth_s
    suth_s: float = 0.368
    integrator: int = AB2            # AB2, or RK3 (synchronous steps only)
    extrapolate_state: bool = False  # AT ghosts: q of the extrapolated state, not the extrapolated q
    mixed_central: bool = False      # mixed terms: central stencil over the neighbour's gradient

    @property
    def scheme(self):
        return Scheme(self.order)

    @property
    def nloc(self):
        return tuple(self.n[d] // self.pes[d] for d in range(3))

    @property
    def dx(self):
        return tuple(2.0 * math.pi / self.n[d] for d in range(3))

    @property
    def n_levels(self):
        """Time levels held: n, n-1, ..., n-(L+T_l-1)  (Sec. 3.1: L + T_l)."""
        return self.max_delay + self.scheme.T

    @property
    def n_pes(self):
        return self.pes[0] * self.pes[1] * self.pes[2]


# --------------------------------------------------------------------------
# geometry: arrays are indexed [z, y, x]; direction d = 0, 1, 2 is x, y, z
# --------------------------------------------------------------------------
def _axis(d):
    return 2 - d


def _coord(cfg, d):
    """Index along direction d, shaped to broadcast against a [z, y, x] field."""
    shape = [1, 1, 1]
    shape[_axis(d)] = cfg.n[d]
    return np.arange(cfg.n[d]).reshape(shape)


def pe_index_field(cfg):
    """PE number p = (pz * Py + py) * Px + px of every grid point."""
    px = _coord(cfg, 0) // cfg.nloc[0]
    py = _coord(cfg, 1) // cfg.nloc[1]
    pz = _coord(cfg, 2) // cfg.nloc[2]
    return np.broadcast_to((pz * cfg.pes[1] + py) * cfg.pes[0] + px,
                           (cfg.n[2], cfg.n[1], cfg.n[0]))


def boundary_fraction(cfg):
    """N_B / N_T per PE, Eqs. (NT), (NI), (NB) (M = order / 2)."""
    M = cfg.scheme.M
    nt = 1
    ni = 1
    for d in range(3):
        nt *= cfg.nloc[d]
        ni *= cfg.nloc[d] - 2 * M
    return (nt - ni) / nt


# --------------------------------------------------------------------------
# delay map (Sec. 3.1, Algorithms 1 and 2)
# --------------------------------------------------------------------------
def delay_map(cfg, step, mode):
    """Delays k[p, f] for step n; faces f = x-, x+, y-, y+, z-, z+."""
    P = cfg.n_pes
    k = np.zeros((P, 6), dtype=np.int64)
    n0 = cfg.n_levels                       # synchronous start-up: L + T_l steps
    if mode == SYNC or step < n0:
        return k
    if mode == PERIODIC:
        k[:] = (step - n0) % cfg.comm_period
        return k
    if mode == FIXED:                       # worst case of the stability analysis (Sec. 3.2)
        k[:] = cfg.max_delay
        return k
    if mode in (RANDOM, ORDERED):
        p = np.arange(P, dtype=np.uint64)[:, None]
        f = np.arange(6, dtype=np.uint64)[None, :]
        k0, k1 = split_seed(cfg.seed)

        def draw(m):
            w0, _, _, _ = philox4x32_10(np.uint64(m), p, f, np.uint64(DELAY_STREAM_TAG), k0, k1)
            # uniform integer on {0..L}: floor(w * (L+1) / 2^32), exact in integers
            return ((w0.astype(np.uint64) * np.uint64(cfg.max_delay + 1)) >> np.uint64(32)).astype(np.int64)

        if mode == RANDOM:
            return draw(step)
        # ordered: the newest level a PE has received never ages by more than
        # one step per step (its neighbour's messages arrive in order, Alg. 1):
        # k_n = min(d_n, k_{n-1} + 1), k = 0 before n0, d the draws of RANDOM.
        # Unrolled, k_n = min over j of (d_{n-j} + j) and (n - n0 + 1); terms
        # with j > L exceed d_n and cannot be the minimum.
        k = draw(step)
        for j in range(1, min(cfg.max_delay, step - n0) + 1):
            k = np.minimum(k, draw(step - j) + j)
        return np.minimum(k, step - n0 + 1)
    raise ValueError("unknown delay mode")


# --------------------------------------------------------------------------
# primitive variables and differentiated quantities
# --------------------------------------------------------------------------
def primitives(cfg, U):
    """rho, (u, v, w), p, T from conserved (rho, rho u, rho v, rho w, E or rho e)."""
    rho = U[0]
    vel = [U[1] / rho, U[2] / rho, U[3] / rho]
    if cfg.energy_form == ENERGY_INTERNAL:
        p = (cfg.gamma - 1.0) * U[4]
    else:
        ke = 0.5 * rho * (vel[0] ** 2 + vel[1] ** 2 + vel[2] ** 2)
        p = (cfg.gamma - 1.0) * (U[4] - ke)
    T = cfg.gamma * p / rho
    return rho, vel, p, T


def quantity(cfg, U, name):
    """A differentiated quantity evaluated from one time level of U.

    'F{d}{e}': component e of the inviscid flux in direction d
               (rho u_d, rho u_i u_d + p delta_id, (E + p) u_d or rho e u_d);
    'u0','u1','u2': velocity components; 'T': temperature.
    """
    rho, vel, p, T = primitives(cfg, U)
    if name == "T":
        return T
    if name[0] == "u":
        return vel[int(name[1])]
    d, e = int(name[1]), int(name[2])
    if e == 0:
        return U[1 + d]
    if e == 4:
        if cfg.energy_form == ENERGY_INTERNAL:
            return U[4] * vel[d]
        return (U[4] + p) * vel[d]
    i = e - 1
    return U[1 + i] * vel[d] + (p if i == d else 0.0)


# --------------------------------------------------------------------------
# AT derivatives (Eq. (at), Table B)
# --------------------------------------------------------------------------
def _face_delay_field(cfg, delays, d):
    """Per point: delay of the face its d-stencil crosses (0 if it crosses none)."""
    li = _coord(cfg, d) % cfg.nloc[d]
    pe = pe_index_field(cfg)
    k_left = delays[pe, 2 * d]
    k_right = delays[pe, 2 * d + 1]
    M = cfg.scheme.M
    k = np.where(li < M, k_left, np.where(li >= cfg.nloc[d] - M, k_right, 0))
    return np.broadcast_to(k, pe.shape)


def at_derivative(cfg, qlevels, d, delays, order, qext=None):
    """First (order=1) or second (order=2) AT derivative in direction d.

    qlevels[l] is the quantity at level n-l.  Literal Table B: the standard
    stencil is evaluated once per l = 0 .. T_l-1 with the points outside the
    PE taken at level n-k-l, and the T_l results are weighted by w_l(k).
    Points inside the PE always use level n.  A direction with one PE is a
    plain periodic stencil at level n.

    qext (the other reading of what Table B extrapolates): qext[k] is the
    quantity of the state extrapolated to level n from the levels n-k-l,
    q(sum_l w_l(k) U^{n-k-l}); the points outside the PE then take qext[k]
    and the stencil is evaluated once.
    """
    sc = cfg.scheme
    stencil, denom = (sc.d1, sc.d1_den * cfg.dx[d]) if order == 1 else \
                     (sc.d2, sc.d2_den * cfg.dx[d] ** 2)
    ax = _axis(d)
    if cfg.pes[d] == 1:
        out = np.zeros_like(qlevels[0])
        for off, c in stencil:
            out += c * np.roll(qlevels[0], -off, axis=ax)
        return out / denom
    nloc = cfg.nloc[d]
    li = _coord(cfg, d) % nloc
    kf = _face_delay_field(cfg, delays, d)
    if qext is not None:
        X = np.stack(qext)                      # [delay k, z, y, x]
        out = np.zeros_like(qlevels[0])
        for off, c in stencil:
            inside = (li + off >= 0) & (li + off < nloc)
            q0 = np.roll(qlevels[0], -off, axis=ax)
            shifted = np.roll(X, -off, axis=ax + 1)
            qk = np.take_along_axis(shifted, np.broadcast_to(kf, kf.shape)[None], axis=0)[0]
            out += c * np.where(inside, q0, qk)
        return out / denom
    Q = np.stack(qlevels)                       # [level, z, y, x]
    out = np.zeros_like(qlevels[0])
    wtab = np.array([sc.weights(k) for k in range(int(np.max(kf)) + 1)])   # Table B weights per delay
    for l in range(sc.T):
        w = wtab[kf, l]
        S = np.zeros_like(qlevels[0])
        for off, c in stencil:
            inside = (li + off >= 0) & (li + off < nloc)
            level = np.where(inside, 0, kf + l)
            shifted = np.roll(Q, -off, axis=ax + 1)  # shifted[:, ..., i] = Q[:, ..., i+off]
            val = np.take_along_axis(shifted, np.broadcast_to(level, kf.shape)[None], axis=0)[0]
            S += c * val
        out += w * S
    return out / denom


def _central_fits(cfg, d):
    """True where the central d-stencil stays inside the PE (or d has one PE)."""
    li = _coord(cfg, d) % cfg.nloc[d]
    if cfg.pes[d] == 1:
        return np.ones_like(li, dtype=bool)
    M = cfg.scheme.M
    return (li >= M) & (li <= cfg.nloc[d] - 1 - M)


def _apply(f, stencil, ax):
    out = np.zeros_like(f)
    for off, c in stencil:
        out += c * np.roll(f, -off, axis=ax)
    return out


def pe_local_d1(cfg, g, d):
    """PE-local first derivative of the scheme's order: central where it fits
    inside the PE, one-sided at the M points next to each PE face (no data
    from other PEs is read)."""
    sc = cfg.scheme
    ax = _axis(d)
    den = sc.d1_den * cfg.dx[d]
    out = _apply(g, sc.d1, ax)
    if cfg.pes[d] == 1:
        return out / den
    nloc = cfg.nloc[d]
    li = _coord(cfg, d) % nloc
    for j in list(range(sc.M)) + list(range(nloc - sc.M, nloc)):
        out = np.where(li == j, _apply(g, sc.one_sided(j, nloc), ax), out)
    return out / den


def mixed_derivative(cfg, grad_b, grad_a, a, b):
    """d/dx_a (d f/dx_b) by the three-step rule of Sec. 2.1.

    grad_b = AT first derivative of f in b, grad_a = AT first derivative of f in
    a (both already computed with AT stencils at PE faces).  At points whose
    a- and b-stencils both fit inside the PE the standard central derivative in
    a of grad_b is used.  At the other (boundary) points the PE-local
    derivative in a of grad_b and the PE-local derivative in b of grad_a are
    averaged.
    """
    sc = cfg.scheme
    interior = _central_fits(cfg, a) & _central_fits(cfg, b)
    central = _apply(grad_b, sc.d1, _axis(a)) / (sc.d1_den * cfg.dx[a])
    boundary = 0.5 * (pe_local_d1(cfg, grad_b, a) + pe_local_d1(cfg, grad_a, b))
    return np.where(interior, central, boundary)


def mixed_central(cfg, grad_b, qb, a, b, delays):
    """d/dx_a (d f/dx_b) by the central a-stencil at every point: the other
    reading of the mixed terms at PE faces.

    Stencil points inside the PE take the AT first derivative grad_b there.
    A point across an a-face of delay k takes the neighbour's b-derivative
    extrapolated to level n with the Table B weights: qb[k] is that field,
    sum_l w_l(k) D_b f^{n-k-l} (or D_b of f of the extrapolated state), D_b
    being the plain central stencil of the whole level.  Without delays this
    is the central D_a D_b of the single-PE scheme.
    """
    sc = cfg.scheme
    ax = _axis(a)
    den = sc.d1_den * cfg.dx[a]
    if cfg.pes[a] == 1:
        return _apply(grad_b, sc.d1, ax) / den
    nloc = cfg.nloc[a]
    li = _coord(cfg, a) % nloc
    kf = _face_delay_field(cfg, delays, a)
    X = np.stack(qb)                            # [delay k, z, y, x]
    out = np.zeros_like(grad_b)
    for off, c in sc.d1:
        inside = (li + off >= 0) & (li + off < nloc)
        g_in = np.roll(grad_b, -off, axis=ax)
        g_out = np.take_along_axis(np.roll(X, -off, axis=ax + 1), np.broadcast_to(kf, kf.shape)[None], axis=0)[0]
        out += c * np.where(inside, g_in, g_out)
    return out / den


def ghost_gradients(cfg, flevels, b):
    """Per delay k = 0 .. L: sum_l w_l(k) D_b f^{n-k-l}, D_b the plain
    central first derivative of a whole level (flevels[l] = f at level n-l)."""
    sc = cfg.scheme
    den = sc.d1_den * cfg.dx[b]
    D = [_apply(f, sc.d1, _axis(b)) / den for f in flevels]
    out = []
    for k in range(cfg.max_delay + 1):
        w = sc.weights(k)
        g = w[0] * D[k]
        for l in range(1, sc.T):
            g = g + w[l] * D[k + l]
        out.append(g)
    return out


# --------------------------------------------------------------------------
# forcing (Sec. 4.2): solenoidal, |kappa| <= kappa_f
# --------------------------------------------------------------------------
def forcing_modes(kf):
    """Half set of integer wavevectors 0 < |k| <= kf: k_x > 0, or k_x = 0 and
    k_y > 0, or k_x = k_y = 0 and k_z > 0.  Order: k_z outer, k_x inner."""
    K = int(math.floor(kf))
    modes = []
    for kz in range(-K, K + 1):
        for ky in range(-K, K + 1):
            for kx in range(-K, K + 1):
                k2 = kx * kx + ky * ky + kz * kz
                if k2 == 0 or k2 > kf * kf + 1e-12:
                    continue
                if kx > 0 or (kx == 0 and ky > 0) or (kx == 0 and ky == 0 and kz > 0):
                    modes.append((kx, ky, kz))
    return modes


def forcing_noise(cfg, step, modes):
    """Complex standard normals xi[m, c] (Box-Muller on Philox words 0, 1)."""
    k0, k1 = split_seed(cfg.f_seed)
    m = np.arange(len(modes), dtype=np.uint64)[:, None]
    c = np.arange(3, dtype=np.uint64)[None, :]
    w0, w1, _, _ = philox4x32_10(np.uint64(step), m, c, np.uint64(FORCING_STREAM_TAG), k0, k1)
    u1 = (w0.astype(np.float64) + 0.5) * 2.0 ** -32
    u2 = (w1.astype(np.float64) + 0.5) * 2.0 ** -32
    r = np.sqrt(-2.0 * np.log(u1))
    return r * np.cos(2.0 * math.pi * u2) + 1j * r * np.sin(2.0 * math.pi * u2)


def solenoidal_projection(modes, v):
    """v - k (k . v) / |k|^2 for each mode."""
    k = np.array(modes, dtype=np.float64)
    kv = np.sum(k * v, axis=1)
    return v - k * (kv / np.sum(k * k, axis=1))[:, None]


def forcing_coefficients(cfg, step):
    """OU coefficients f_hat[m, c] at step n: f^0 = s P(xi^0),
    f^n = a f^{n-1} + s sqrt(1 - a^2) P(xi^n), a = exp(-dt / T_f)."""
    modes = forcing_modes(cfg.kf)
    a = math.exp(-cfg.dt / cfg.f_tcorr)
    b = cfg.f_amp * math.sqrt(1.0 - a * a)
    fh = cfg.f_amp * solenoidal_projection(modes, forcing_noise(cfg, 0, modes))
    for s in range(1, step + 1):
        fh = a * fh + b * solenoidal_projection(modes, forcing_noise(cfg, s, modes))
    return fh


def forcing_field(cfg, fhat):
    """f_c(x) = sum over the half set of 2 Re(f_hat[m, c] exp(i k . x))."""
    modes = forcing_modes(cfg.kf)
    x = [_coord(cfg, d) * cfg.dx[d] for d in range(3)]
    f = [np.zeros((cfg.n[2], cfg.n[1], cfg.n[0])) for _ in range(3)]
    for m, (kx, ky, kz) in enumerate(modes):
        phase = np.exp(1j * (kx * x[0] + ky * x[1] + kz * x[2]))
        for c in range(3):
            f[c] += 2.0 * np.real(fhat[m, c] * phase)
    return f


# --------------------------------------------------------------------------
# transport coefficients (Sec. 2)
# --------------------------------------------------------------------------
def viscosity(cfg, T):
    """mu(T) and d mu / dT: power law mu0 T^omega, or Sutherland
    mu0 T^(3/2) (1 + S) / (T + S)."""
    if cfg.visc_law == VISC_SUTHERLAND:
        S = cfg.suth_s
        mu = cfg.mu0 * T ** 1.5 * (1.0 + S) / (T + S)
        return mu, mu * (1.5 / T - 1.0 / (T + S))
    mu = cfg.mu0 * T ** cfg.visc_exp
    return mu, cfg.visc_exp * mu / T


# --------------------------------------------------------------------------
# right-hand side
# --------------------------------------------------------------------------
def rhs(cfg, levels, delays, fhat=None, return_aux=False):
    """R(U^n) for the conserved variables.

    levels[l] = U^{n-l} for l = 0 .. L+T_l-1, each shaped [5, nz, ny, nx].
    delays[p, f] = this step's delay map.  fhat = forcing coefficients (or None).
    """
    nlev = len(levels)
    g = cfg.gamma

    def q_levels(name):
        return [quantity(cfg, levels[l], name) for l in range(nlev)]

    # the state extrapolated to level n for every delay k (the other reading
    # of Table B's weights): U_k = sum_l w_l(k) U^{n-k-l}
    if cfg.extrapolate_state:
        sc = cfg.scheme
        Uext = []
        for k in range(cfg.max_delay + 1):
            w = sc.weights(k)
            Uk = w[0] * levels[k]
            for l in range(1, sc.T):
                Uk = Uk + w[l] * levels[k + l]
            Uext.append(Uk)

    def q_ext(name):
        return [quantity(cfg, Uk, name) for Uk in Uext] if cfg.extrapolate_state else None

    def D1(name, d):
        return at_derivative(cfg, q_levels(name), d, delays, 1, q_ext(name))

    def D2(name, d):
        return at_derivative(cfg, q_levels(name), d, delays, 2, q_ext(name))

    rho, vel, p, T = primitives(cfg, levels[0])
    R = np.zeros_like(levels[0])

    # inviscid part: - sum_j d/dx_j F_j
    for d in range(3):
        for e in range(5):
            R[e] -= D1("F%d%d" % (d, e), d)

    # first derivatives A[i][j] = d u_i / d x_j and dT/dx_j (AT at faces)
    A = [[D1("u%d" % i, j) for j in range(3)] for i in range(3)]
    dT = [D1("T", j) for j in range(3)]
    # second derivatives d^2 u_i / d x_j^2 and d^2 T / d x_j^2
    D2u = [[D2("u%d" % i, j) for j in range(3)] for i in range(3)]
    lap_u = [D2u[i][0] + D2u[i][1] + D2u[i][2] for i in range(3)]
    lap_T = D2("T", 0) + D2("T", 1) + D2("T", 2)
    theta = A[0][0] + A[1][1] + A[2][2]

    # d theta / d x_i = d^2 u_i / d x_i^2 + sum_{k != i} d/dx_i (d u_k / d x_k)
    grad_theta = []
    for i in range(3):
        s = D2u[i][i].copy()
        for k in range(3):
            if k != i:
                # mixed d/dx_i (d u_k/dx_k): grad in b=k is A[k][k], grad in a=i is A[k][i]
                if cfg.mixed_central:
                    name = "u%d" % k
                    if cfg.extrapolate_state:
                        den = cfg.scheme.d1_den * cfg.dx[k]
                        qb = [_apply(f, cfg.scheme.d1, _axis(k)) / den for f in q_ext(name)]
                    else:
                        qb = ghost_gradients(cfg, q_levels(name), k)
                    s = s + mixed_central(cfg, A[k][k], qb, i, k, delays)
                else:
                    s = s + mixed_derivative(cfg, A[k][k], A[k][i], i, k)
        grad_theta.append(s)

    mu, dmu_dT = viscosity(cfg, T)
    dmu = [dmu_dT * dT[j] for j in range(3)]
    cp = 1.0 / (g - 1.0)
    kappa = mu * cp / cfg.prandtl
    dkappa = [dmu[j] * cp / cfg.prandtl for j in range(3)]

    delta = lambda i, j: 1.0 if i == j else 0.0
    sigma = [[mu * (A[i][j] + A[j][i] - (2.0 / 3.0) * delta(i, j) * theta) for j in range(3)]
             for i in range(3)]
    S = [[0.5 * (A[i][j] + A[j][i]) for j in range(3)] for i in range(3)]

    # viscous momentum term V_i = d sigma_ij / d x_j, expanded
    V = []
    for i in range(3):
        v = mu * (lap_u[i] + grad_theta[i] / 3.0)
        for j in range(3):
            v = v + dmu[j] * (A[i][j] + A[j][i] - (2.0 / 3.0) * delta(i, j) * theta)
        V.append(v)

    if fhat is not None:
        f = forcing_field(cfg, fhat)
    else:
        f = [np.zeros_like(rho)] * 3

    for i in range(3):
        R[1 + i] += V[i] + rho * f[i]
    sigS = sum(sigma[i][j] * S[i][j] for i in range(3) for j in range(3))
    heat = kappa * lap_T + sum(dkappa[j] * dT[j] for j in range(3))
    if cfg.energy_form == ENERGY_INTERNAL:
        # Eq. (ie): -p theta + sigma_ij S_ij + d(k dT/dx_j)/dx_j
        R[4] += -p * theta + sigS + heat
    else:
        R[4] += (sum(vel[i] * V[i] for i in range(3)) + sigS + heat
                 + sum(rho * f[i] * vel[i] for i in range(3)))
    if not return_aux:
        return R
    aux = dict(rho=rho, vel=vel, p=p, T=T, A=A, theta=theta, sigS=sigS, f=f)
    return R, aux


# --------------------------------------------------------------------------
# statistics (volume averages, FP64)
# --------------------------------------------------------------------------
def statistics(cfg, U, aux):
    rho, vel, p, T, A = aux["rho"], aux["vel"], aux["p"], aux["T"], aux["A"]
    mean = lambda a: float(np.mean(a))
    u2 = vel[0] ** 2 + vel[1] ** 2 + vel[2] ** 2
    c = np.sqrt(T)                       # c^2 = gamma p / rho = T
    m2 = np.mean([mean(A[i][i] ** 2) for i in range(3)])
    m3 = np.mean([mean(A[i][i] ** 3) for i in range(3)])
    m4 = np.mean([mean(A[i][i] ** 4) for i in range(3)])
    om = [A[2][1] - A[1][2], A[0][2] - A[2][0], A[1][0] - A[0][1]]
    wave = max(float(np.max(np.abs(vel[d]) + c)) for d in range(3))
    return dict(
        mass=mean(U[0]), mom=[mean(U[1]), mean(U[2]), mean(U[3])], energy=mean(U[4]),
        tke=mean(0.5 * rho * u2), dissipation=mean(aux["sigS"]),
        grad_m2=m2, grad_m3=m3, grad_m4=m4,
        skewness=m3 / m2 ** 1.5, flatness=m4 / m2 ** 2,
        enstrophy=mean(om[0] ** 2 + om[1] ** 2 + om[2] ** 2),
        pressure_dilatation=mean(p * aux["theta"]),
        forcing_power=mean(rho * (aux["f"][0] * vel[0] + aux["f"][1] * vel[1] + aux["f"][2] * vel[2])),
        urms=math.sqrt(mean(u2) / 3.0), mach_t=math.sqrt(mean(u2)) / mean(c),
        max_wave_speed=wave, min_rho=float(np.min(rho)), min_p=float(np.min(p)))


def max_wave_speed(cfg, U):
    """max over points and directions of |u_d| + c."""
    rho, vel, p, T = primitives(cfg, U)
    c = np.sqrt(T)
    return max(float(np.max(np.abs(vel[d]) + c)) for d in range(3))


def dt_from_cfl(cfg, U, cfl):
    """Fixed time step from the convective CFL at t = 0 (Sec. 2.2): dt = r_c dx / s."""
    rho, vel, p, T = primitives(cfg, U)
    c = np.sqrt(T)
    s = max(float(np.max((np.abs(vel[d]) + c) / cfg.dx[d])) for d in range(3))
    return cfl / s


# --------------------------------------------------------------------------
# time stepping (Eq. (time_ab), AB2)
# --------------------------------------------------------------------------
def ab2_update(U, R, R_prev, dt):
    """u^{n+1} = u^n + dt (3/2 f^n - 1/2 f^{n-1}); forward Euler when no f^{n-1}."""
    if R_prev is None:
        return U + dt * R
    return U + dt * (1.5 * R - 0.5 * R_prev)


@dataclass
class Run:
    """Oracle time loop: holds U^n .. U^{n-L-T_l+1} in full (levels[0] = U^n)."""
    cfg: Config
    mode: int
    levels: list = field(default_factory=list)
    step_n: int = 0
    R_prev: object = None

    @classmethod
    def start(cls, cfg, U0, mode, step=0, history=None):
        """All stored levels equal U0 (the synchronous start-up fill), unless an
        explicit history [U^n, U^{n-1}, ...] is given."""
        if history is None:
            levels = [np.array(U0, dtype=np.float64) for _ in range(cfg.n_levels)]
        else:
            levels = [np.array(h, dtype=np.float64) for h in history]
            levels += [levels[-1]] * (cfg.n_levels - len(levels))
        return cls(cfg=cfg, mode=mode, levels=levels, step_n=step)

    def delays(self):
        return delay_map(self.cfg, self.step_n, self.mode)

    def fhat(self):
        return forcing_coefficients(self.cfg, self.step_n) if self.cfg.forcing else None

    def rhs(self, return_aux=False):
        return rhs(self.cfg, self.levels, self.delays(), self.fhat(), return_aux)

    def step(self):
        if self.cfg.integrator == RK3:
            return self.step_rk3()
        R = self.rhs()
        U_new = ab2_update(self.levels[0], R, self.R_prev, self.cfg.dt)
        self.levels = [U_new] + self.levels[:-1]
        self.R_prev = R
        self.step_n += 1
        return U_new

    def step_rk3(self):
        """Three low-storage RK stages from U^n, each with the forcing of step
        n and no delays."""
        if self.mode != SYNC:
            raise ValueError("RK3 steps are synchronous")
        fhat = self.fhat()
        zero = np.zeros((self.cfg.n_pes, 6), dtype=np.int64)
        U = self.levels[0].copy()
        dU = np.zeros_like(U)
        for s in range(3):
            R = rhs(self.cfg, [U] + self.levels[1:], zero, fhat)
            dU = RK3_A[s] * dU + self.cfg.dt * R
            U = U + RK3_B[s] * dU
        self.levels = [U] + self.levels[:-1]
        self.step_n += 1
        return U
