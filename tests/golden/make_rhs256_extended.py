"""Writes rhs256_sampled_extended.txt: the right-hand side of the 256^3
benchmark workload (8x8x8 PEs of 32^3, random delays with L = 2, step 17) at
the sampled points of the full-size GPU parity test, evaluated by the
oracle's brute-force pointwise evaluator twice -- in FP64 as it stands, and
in 40-digit arithmetic (mpmath) with exact stencil coefficients and grid
spacing -- from the same seeded FP64 inputs.

The difference between the two is the FP64 oracle's own rounding at those
points: the floor that any FP64 evaluation of the same sums in another order
(the CUDA path) is expected to reach, and the basis of the FP64 tolerance of
that test.  Calls only oracle/ and the seeded input generator.

Usage: python tests/golden/make_rhs256_extended.py   (about a minute or two)
"""
import os
import sys

import mpmath
import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import ns  # noqa: E402
from oracle.pointwise import PointOracle  # noqa: E402
from tests.sampling import FULL_STEP, full_size_history, full_size_points  # noqa: E402

mpmath.mp.dps = 40
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "rhs256_sampled_extended.txt")


class ExtendedPointOracle(PointOracle):
    """The pointwise evaluator with 40-digit values, exact stencil weights
    (integers over the stencil denominator times the exact dx = 2 pi / N)."""

    def __init__(self, *a, **kw):
        super().__init__(*a, **kw)
        self.dxm = [2 * mpmath.pi / self.cfg.n[d] for d in range(3)]

    def U(self, l, pos):
        pos = self._wrap(pos)
        key = (l, pos)
        if key not in self._ucache:
            lv = self.level(l)
            x, y, z = pos
            self._ucache[key] = [mpmath.mpf(float(lv[v, z, y, x])) for v in range(5)]
        return self._ucache[key]

    def terms(self, pos, d, order):
        """The same (offset, level, weight) list as the FP64 evaluator, with
        the weights w_l(k) c / (den dx^order) formed exactly."""
        cfg, sc = self.cfg, self.sc
        stencil, den = (sc.d1, sc.d1_den) if order == 1 else (sc.d2, sc.d2_den)
        denom = mpmath.mpf(den) * self.dxm[d] ** order
        if cfg.pes[d] == 1:
            return [(off, 0, mpmath.mpf(c) / denom) for off, c in stencil]
        nloc, li, p = cfg.nloc[d], self.local(pos, d), self.pe_of(pos)
        k = 0
        if li < sc.M:
            k = int(self.delays[p][2 * d])
        elif li >= nloc - sc.M:
            k = int(self.delays[p][2 * d + 1])
        w = sc.weights(k)
        return [(off, 0 if 0 <= li + off < nloc else k + l, mpmath.mpf(w[l]) * c / denom)
                for l in range(sc.T) for off, c in stencil]

    def _apply_d1(self, stencil, gfun, pos, d):
        s = mpmath.mpf(0)
        for off, c in stencil:
            p2 = list(pos)
            p2[d] += off
            s += c * gfun(tuple(p2))
        return s / (self.sc.d1_den * self.dxm[d])


def main():
    cfg, hist = full_size_history()
    delays = ns.delay_map(cfg, FULL_STEP, ns.RANDOM)
    pts = full_size_points()
    po = PointOracle(cfg, lambda l: hist[l], delays)
    pe = ExtendedPointOracle(cfg, lambda l: hist[l], delays)
    rows = []
    for i, p in enumerate(pts):
        r64 = po.rhs(p)
        rex = pe.rhs(p)
        rows.append((p, r64, rex))
        if i % 20 == 0:
            print("%d / %d" % (i, len(pts)), flush=True)
    ext = np.array([[float(v) for v in r[2]] for r in rows])
    f64 = np.array([r[1] for r in rows])
    scale = np.max(np.abs(ext), axis=0)
    floor = np.max(np.abs(f64 - ext), axis=0) / scale
    with open(OUT, "w") as f:
        f.write("# RHS of the 256^3 workload (8x8x8 PEs, random delays L = 2, step 17) at the sampled points of\n")
        f.write("# tests/test_gpu_parity.py::test_full_size_sampled_parity, written by make_rhs256_extended.py.\n")
        f.write("# columns: x y z, then for v = 0..4 the 40-digit value (rounded to 20 digits) and the FP64\n")
        f.write("# oracle's value.  FP64 oracle floor per variable (max |fp64 - ext| / max |ext|):\n")
        f.write("# floor " + " ".join("%.3e" % v for v in floor) + "\n")
        for (p, r64, rex) in rows:
            f.write("%d %d %d " % p + " ".join("%s %r" % (mpmath.nstr(rex[v], 20), float(r64[v])) for v in range(5)) + "\n")
    print("floor per variable:", floor)


if __name__ == "__main__":
    main()
