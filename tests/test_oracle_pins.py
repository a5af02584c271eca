"""Pins of the oracle's mixed-derivative rule (Sec. 2.1) and of its velocity-
gradient moments, skewness and flatness (Sec. 4.1), against facts that do not
come from the oracle itself.

* Mixed rule.  At PE-boundary points the rule averages the PE-local derivative
  in a of the AT derivative in b and the PE-local derivative in b of the AT
  derivative in a, so it is symmetric under exchanging (a, G_b) with
  (b, G_a).  And since every stencil it applies stays inside one PE, with
  G_a = df/dx_a and G_b = df/dx_b of a polynomial f of degree <= 4 per
  direction (4th order; <= 6 at 6th order), it returns d2f/dx_a dx_b exactly
  at every point.  A variant without the average (PE-local D_a(G_b) alone)
  keeps the exactness but fails the symmetry; a variant with the operands
  exchanged (D_a(G_a) and D_b(G_b)) keeps the symmetry but fails exactness.

* Moments.  For u = a sin x + b sin 2x, v = c sin x, w = 0 on a uniform-density,
  uniform-pressure field, the 4th-order first derivative is exact up to the
  modified wavenumber k'(m) = (8 sin(m h) - sin(2 m h)) / (6 h), so
  du/dx = alpha cos x + beta cos 2x with alpha = a k'(1), beta = b k'(2), and
  the grid averages of the trigonometric products are those of the continuum
  (no product here reaches frequency N/2):
      <(du/dx)^2> = (alpha^2 + beta^2)/2,  <(du/dx)^3> = 3 alpha^2 beta / 4,
      <(du/dx)^4> = 3/8 alpha^4 + 3/2 alpha^2 beta^2 + 3/8 beta^4.
  The oracle's moments average over the three diagonal gradients, two of
  which vanish here.  A variant that averages |A_ii|^3 instead of A_ii^3, or
  that drops the average over components, fails.
"""
import math

import numpy as np
import pytest

from oracle import ns
from oracle.pointwise import PointOracle


# ---------------------------------------------------------------------------
# mixed-derivative rule
# ---------------------------------------------------------------------------
def _boundary_mask(cfg, a, b):
    m = ~(ns._central_fits(cfg, a) & ns._central_fits(cfg, b))
    return np.broadcast_to(m, (cfg.n[2], cfg.n[1], cfg.n[0]))


def _unaveraged(cfg, grad_b, grad_a, a, b):
    """Planted mistake: the PE-local derivative in a of G_b alone."""
    sc = cfg.scheme
    interior = ns._central_fits(cfg, a) & ns._central_fits(cfg, b)
    central = ns._apply(grad_b, sc.d1, ns._axis(a)) / (sc.d1_den * cfg.dx[a])
    return np.where(interior, central, ns.pe_local_d1(cfg, grad_b, a))


def _swapped(cfg, grad_b, grad_a, a, b):
    """Planted mistake: each direction's derivative of its own gradient."""
    sc = cfg.scheme
    interior = ns._central_fits(cfg, a) & ns._central_fits(cfg, b)
    central = ns._apply(grad_b, sc.d1, ns._axis(a)) / (sc.d1_den * cfg.dx[a])
    boundary = 0.5 * (ns.pe_local_d1(cfg, grad_a, a) + ns.pe_local_d1(cfg, grad_b, b))
    return np.where(interior, central, boundary)


def _smooth_field(cfg, seed):
    """A smooth, non-polynomial periodic field (a few random Fourier modes)."""
    rng = np.random.default_rng(seed)
    z, y, x = np.meshgrid(*[np.arange(cfg.n[d]) * cfg.dx[d] for d in (2, 1, 0)], indexing="ij")
    f = np.zeros(z.shape)
    for _ in range(6):
        k = rng.integers(-3, 4, size=3)
        f += rng.normal() * np.cos(k[0] * x + k[1] * y + k[2] * z + rng.uniform(0, 2 * math.pi))
    return f


def _pe_polynomial(cfg, a, b, deg):
    """f = P(s_a) Q(s_b) with s_d the coordinate relative to the PE origin, and
    its exact first derivatives and mixed derivative."""
    rng = np.random.default_rng(100 + 10 * a + b + deg)
    p = rng.normal(size=deg + 1)
    q = rng.normal(size=deg + 1)
    s = [(ns._coord(cfg, d) % cfg.nloc[d]) * cfg.dx[d] * np.ones((cfg.n[2], cfg.n[1], cfg.n[0])) for d in range(3)]
    P, Pp = np.polyval(p, s[a]), np.polyval(np.polyder(p), s[a])
    Q, Qp = np.polyval(q, s[b]), np.polyval(np.polyder(q), s[b])
    return P * Qp, Pp * Q, Pp * Qp        # G_b, G_a, d2f / dx_a dx_b


CASES = [
    # (grid, PEs, order)
    ((32, 32, 16), (4, 4, 2), 4),
    ((24, 20, 28), (3, 2, 4), 4),
    ((42, 28, 21), (3, 2, 3), 6),
]


@pytest.mark.parametrize("n,pes,order", CASES)
def test_mixed_rule_symmetric_at_boundary_points(n, pes, order):
    cfg = ns.Config(n=n, pes=pes, order=order)
    G1, G2 = _smooth_field(cfg, 1), _smooth_field(cfg, 2)
    for a, b in ((0, 1), (0, 2), (1, 2)):
        mask = _boundary_mask(cfg, a, b)
        assert mask.any() and not mask.all()
        m_ab = ns.mixed_derivative(cfg, G1, G2, a, b)
        m_ba = ns.mixed_derivative(cfg, G2, G1, b, a)
        scale = np.max(np.abs(m_ab))
        assert np.max(np.abs(m_ab - m_ba)[mask]) <= 1e-13 * scale
        # the planted mistake breaks the symmetry by far more than rounding
        u_ab = _unaveraged(cfg, G1, G2, a, b)
        u_ba = _unaveraged(cfg, G2, G1, b, a)
        assert np.max(np.abs(u_ab - u_ba)[mask]) > 1e-3 * scale


@pytest.mark.parametrize("n,pes,order", CASES)
def test_mixed_rule_exact_on_pe_polynomials(n, pes, order):
    cfg = ns.Config(n=n, pes=pes, order=order)
    deg = 4 if order == 4 else 6
    for a, b in ((0, 1), (0, 2), (1, 2), (2, 0)):
        Gb, Ga, exact = _pe_polynomial(cfg, a, b, deg)
        scale = np.max(np.abs(exact))
        got = ns.mixed_derivative(cfg, Gb, Ga, a, b)
        assert np.max(np.abs(got - exact)) <= 1e-11 * scale
        # exchanging the operands is a plausible slip: it is not exact
        bad = _swapped(cfg, Gb, Ga, a, b)
        assert np.max(np.abs(bad - exact)) > 1e-2 * scale
    # one degree more is not exact either (the pin has a sharp edge)
    Gb, Ga, exact = _pe_polynomial(cfg, 0, 1, deg + 1)
    got = ns.mixed_derivative(cfg, Gb, Ga, 0, 1)
    assert np.max(np.abs(got - exact)) > 1e-6 * np.max(np.abs(exact))


class _GradOracle(PointOracle):
    """The brute-force evaluator's mixed rule with prescribed gradients."""

    def __init__(self, cfg, grads):
        super().__init__(cfg, level=None, delays=None)
        self.grads = grads

    def grad(self, i, j, pos):
        x, y, z = self._wrap(pos)
        return float(self.grads[j][z, y, x])


@pytest.mark.parametrize("n,pes,order", CASES[:1] + CASES[2:])
def test_pointwise_mixed_rule_pins(n, pes, order):
    cfg = ns.Config(n=n, pes=pes, order=order)
    deg = 4 if order == 4 else 6
    a, b = 0, 2
    Gb, Ga, exact = _pe_polynomial(cfg, a, b, deg)
    grads = {a: Ga, b: Gb, 1: np.zeros_like(Ga)}
    po = _GradOracle(cfg, grads)
    rng = np.random.default_rng(5)
    mask = _boundary_mask(cfg, a, b)
    zs, ys, xs = np.nonzero(mask)
    pick = rng.choice(len(xs), size=40, replace=False)
    scale = np.max(np.abs(exact))
    for i in pick:
        pos = (int(xs[i]), int(ys[i]), int(zs[i]))
        assert abs(po.mixed(0, a, b, pos) - exact[pos[2], pos[1], pos[0]]) <= 1e-11 * scale
    # symmetry on smooth non-polynomial gradients at the same points
    G1, G2 = _smooth_field(cfg, 3), _smooth_field(cfg, 4)
    p1 = _GradOracle(cfg, {a: G2, b: G1, 1: G1})
    for i in pick:
        pos = (int(xs[i]), int(ys[i]), int(zs[i]))
        assert abs(p1.mixed(0, a, b, pos) - p1.mixed(0, b, a, pos)) <= 1e-13 * max(1.0, np.max(np.abs(G1)))


# ---------------------------------------------------------------------------
# velocity-gradient moments, skewness, flatness
# ---------------------------------------------------------------------------
def _wave_state(cfg, a, b, c):
    N = cfg.n[0]
    x = np.arange(N) * cfg.dx[0]
    U = np.zeros((5,) + (cfg.n[2], cfg.n[1], cfg.n[0]))
    U[0] = 1.0
    U[1] = (a * np.sin(x) + b * np.sin(2 * x))[None, None, :]
    U[2] = (c * np.sin(x))[None, None, :]
    U[4] = (1.0 / cfg.gamma) / (cfg.gamma - 1) + 0.5 * (U[1] ** 2 + U[2] ** 2)
    return U


def _closed_form(cfg, a, b, c):
    h = cfg.dx[0]
    kp = lambda m: (8 * math.sin(m * h) - math.sin(2 * m * h)) / (6 * h)
    al, be = a * kp(1), b * kp(2)
    m2 = (al ** 2 + be ** 2) / 2 / 3
    m3 = 3 * al ** 2 * be / 4 / 3
    m4 = (3 / 8 * al ** 4 + 1.5 * al ** 2 * be ** 2 + 3 / 8 * be ** 4) / 3
    g = c * kp(1)                                   # dv/dx = g cos x
    eps = cfg.mu0 * (4.0 / 3.0 * (al ** 2 + be ** 2) / 2 + g ** 2 / 2)
    return dict(grad_m2=m2, grad_m3=m3, grad_m4=m4, skewness=m3 / m2 ** 1.5, flatness=m4 / m2 ** 2,
                tke=(a * a + b * b + c * c) / 4, enstrophy=g ** 2 / 2, dissipation=eps)


def _abs_cube_variant(cfg, U, aux):
    """Planted mistake: <|A_ii|^3> for the third moment."""
    st = ns.statistics(cfg, U, aux)
    A = aux["A"]
    m3 = np.mean([float(np.mean(np.abs(A[i][i]) ** 3)) for i in range(3)])
    st["grad_m3"], st["skewness"] = m3, m3 / st["grad_m2"] ** 1.5
    return st


def _one_component_variant(cfg, U, aux):
    """Planted mistake: moments of du/dx alone (no average over components)."""
    st = ns.statistics(cfg, U, aux)
    A = aux["A"]
    for k, pw in (("grad_m2", 2), ("grad_m3", 3), ("grad_m4", 4)):
        st[k] = float(np.mean(A[0][0] ** pw))
    st["skewness"] = st["grad_m3"] / st["grad_m2"] ** 1.5
    st["flatness"] = st["grad_m4"] / st["grad_m2"] ** 2
    return st


@pytest.mark.parametrize("N", [16, 32])
def test_gradient_moments_skewness_flatness_closed_form(N):
    cfg = ns.Config(n=(N, N, 8), mu0=0.01, visc_exp=0.0)
    a, b, c = 0.07, -0.05, 0.03
    U = _wave_state(cfg, a, b, c)
    R, aux = ns.rhs(cfg, [U] * cfg.n_levels, np.zeros((1, 6), dtype=int), return_aux=True)
    want = _closed_form(cfg, a, b, c)
    st = ns.statistics(cfg, U, aux)
    for k, v in want.items():
        assert abs(st[k] - v) <= 1e-12 * abs(v), (k, st[k], v)
    # S and F are far from the Gaussian 0 and 3: the field is strongly skewed
    assert st["skewness"] < -0.5 and st["flatness"] > 3.0
    for variant in (_abs_cube_variant, _one_component_variant):
        bad = variant(cfg, U, aux)
        assert any(abs(bad[k] - want[k]) > 1e-3 * abs(want[k]) for k in ("skewness", "flatness")), variant
