"""Finite-difference and Asynchrony-Tolerant (AT) stencil definitions, FP64.

Test infrastructure only (see ``oracle/__init__.py``).

Everything here is a plain restatement of the paper's formulas:

* Standard 4th-order central first / second derivatives: the zero-delay rows
  of the (1,4) / (2,4) entries of Table B (Appendix B), i.e.
  D1 f_i = (f_{i-2} - 8 f_{i-1} + 8 f_{i+1} - f_{i+2}) / (12 dx)
  D2 f_i = (-f_{i-2} + 16 f_{i-1} - 30 f_i + 16 f_{i+1} - f_{i+2}) / (12 dx^2)
  (general form Eq. (du) of Sec. 2).
* AT time weights: every Table B row for 4th order is the standard stencil
  evaluated three times, with the points on the delayed side taken at levels
  n-k, n-k-1, n-k-2, weighted by
  w0 = (k^2+3k+2)/2,  w1 = -(k^2+2k),  w2 = (k^2+k)/2      (Table B, T_l = 3).
  At k = 0 these are (1, 0, 0): the AT stencil reduces to the standard one
  (Sec. 2.1).
* One-sided 4th-order first derivatives used for mixed derivatives at PE
  boundary points (Sec. 2.1, mixed-derivative paragraph; the paper says
  "standard one sided" without the order -- the 4th-order textbook stencils are
  taken here):
  at the first point   (-25, 48, -36, 16, -3)/12   on offsets 0..4
  at the second point  (-3, -10, 18, -6, 1)/12     on offsets -1..3
  and their mirror images at the right end of a PE.
* 6th order (the (1,6) / (2,6) rows of Table B): central
  D1 f_i = (-f_{i-3} + 9 f_{i-2} - 45 f_{i-1} + 45 f_{i+1} - 9 f_{i+2} + f_{i+3}) / (60 dx)
  D2 f_i = (2 f_{i-3} - 27 f_{i-2} + 270 f_{i-1} - 490 f_i + 270 f_{i+1}
            - 27 f_{i+2} + 2 f_{i+3}) / (180 dx^2),
  read four times with the delayed points at levels n-k .. n-k-3 and weights
  w0 = (k^3+6k^2+11k+6)/6, w1 = -(k^3+5k^2+6k)/2, w2 = (k^3+4k^2+3k)/2,
  w3 = -(k^3+3k^2+2k)/6                                    (Table B, T_l = 4).
  Two misprints of the table are read as corrected (the symmetric forms):
  the delayed outermost point of the left-boundary rows is i-3 (printed i+3
  in the rows l >= 1), and the second right-boundary (1,6) row is over 60 dx
  (printed 600 dx).  The one-sided first derivatives of the mixed-derivative
  rule are the 7-point 6th-order textbook stencils (/60 dx) at the first
  three points of a PE and their mirror images at the last three.
"""
import numpy as np

# (offset, coefficient) lists, coefficient multiplies f_{i+offset}; divide by 12 dx.
D1_CENTRAL = ((-2, 1.0), (-1, -8.0), (1, 8.0), (2, -1.0))
# divide by 12 dx^2
D2_CENTRAL = ((-2, -1.0), (-1, 16.0), (0, -30.0), (1, 16.0), (2, -1.0))
# one-sided first derivatives (divide by 12 dx)
D1_FORWARD0 = ((0, -25.0), (1, 48.0), (2, -36.0), (3, 16.0), (4, -3.0))
D1_FORWARD1 = ((-1, -3.0), (0, -10.0), (1, 18.0), (2, -6.0), (3, 1.0))
D1_BACKWARD0 = tuple((-o, -c) for o, c in D1_FORWARD0)     # last point of a PE
D1_BACKWARD1 = tuple((-o, -c) for o, c in D1_FORWARD1)     # second to last point

HALF_WIDTH = 2      # M: stencil points on each side (4th order)
T_LEVELS = 3        # T_l: consecutive time levels an AT stencil reads

# 6th order: central stencils (divide by 60 dx and 180 dx^2)
D1_CENTRAL6 = ((-3, -1.0), (-2, 9.0), (-1, -45.0), (1, 45.0), (2, -9.0), (3, 1.0))
D2_CENTRAL6 = ((-3, 2.0), (-2, -27.0), (-1, 270.0), (0, -490.0), (1, 270.0), (2, -27.0), (3, 2.0))
# one-sided 6th-order first derivatives at the first, second and third point
# of a PE (divide by 60 dx)
D1_FORWARD6 = (
    ((0, -147.0), (1, 360.0), (2, -450.0), (3, 400.0), (4, -225.0), (5, 72.0), (6, -10.0)),
    ((-1, -10.0), (0, -77.0), (1, 150.0), (2, -100.0), (3, 50.0), (4, -15.0), (5, 2.0)),
    ((-2, 2.0), (-1, -24.0), (0, -35.0), (1, 80.0), (2, -30.0), (3, 8.0), (4, -1.0)),
)


def at_weights(k):
    """Table B weights (w0, w1, w2) of the levels n-k, n-k-1, n-k-2 for delay k."""
    k = float(k)
    return ((k * k + 3.0 * k + 2.0) / 2.0,
            -(k * k + 2.0 * k),
            (k * k + k) / 2.0)


def at_weights6(k):
    """Table B weights (w0, w1, w2, w3) of the levels n-k .. n-k-3 for delay k
    (6th-order rows, T_l = 4)."""
    k = float(k)
    return ((k ** 3 + 6.0 * k * k + 11.0 * k + 6.0) / 6.0,
            -(k ** 3 + 5.0 * k * k + 6.0 * k) / 2.0,
            (k ** 3 + 4.0 * k * k + 3.0 * k) / 2.0,
            -(k ** 3 + 3.0 * k * k + 2.0 * k) / 6.0)


class Scheme:
    """The stencil set of one spatial order: half width M, time levels T_l,
    central D1 / D2 with their denominators (times dx, dx^2), the one-sided
    first derivatives at the first M points of a PE (mirrored at the last M)
    and the AT weights."""

    def __init__(self, order):
        if order == 4:
            self.M, self.T = HALF_WIDTH, T_LEVELS
            self.d1, self.d1_den = D1_CENTRAL, 12.0
            self.d2, self.d2_den = D2_CENTRAL, 12.0
            self.forward = (D1_FORWARD0, D1_FORWARD1)
            self.weights = at_weights
        elif order == 6:
            self.M, self.T = 3, 4
            self.d1, self.d1_den = D1_CENTRAL6, 60.0
            self.d2, self.d2_den = D2_CENTRAL6, 180.0
            self.forward = D1_FORWARD6
            self.weights = at_weights6
        else:
            raise ValueError("order must be 4 or 6")
        self.order = order

    def one_sided(self, li, nloc):
        """PE-local first-derivative stencil at local index li (denominator d1_den)."""
        if li < self.M:
            return self.forward[li]
        if li >= nloc - self.M:
            return tuple((-o, -c) for o, c in self.forward[nloc - 1 - li])
        return self.d1


def d1_central_periodic(f, axis, dx):
    """Standard 4th-order central first derivative on a periodic axis."""
    out = np.zeros_like(f)
    for off, c in D1_CENTRAL:
        out += c * np.roll(f, -off, axis=axis)
    return out / (12.0 * dx)


def d2_central_periodic(f, axis, dx):
    """Standard 4th-order central second derivative on a periodic axis."""
    out = np.zeros_like(f)
    for off, c in D2_CENTRAL:
        out += c * np.roll(f, -off, axis=axis)
    return out / (12.0 * dx * dx)
