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
  taken here, the reading recorded in the design notes):
  at the first point   (-25, 48, -36, 16, -3)/12   on offsets 0..4
  at the second point  (-3, -10, 18, -6, 1)/12     on offsets -1..3
  and their mirror images at the right end of a PE.
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


def at_weights(k):
    """Table B weights (w0, w1, w2) of the levels n-k, n-k-1, n-k-2 for delay k."""
    k = float(k)
    return ((k * k + 3.0 * k + 2.0) / 2.0,
            -(k * k + 2.0 * k),
            (k * k + k) / 2.0)


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
