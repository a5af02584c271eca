"""The oracle's brute-force pointwise right-hand side evaluated in 40-digit
arithmetic (mpmath), with exact stencil weights and grid spacing, from the
same FP64 inputs.  Its difference from the FP64 evaluation measures the FP64
oracle's own rounding -- the floor that any FP64 evaluation of the same sums
in another order (the CUDA path) is expected to reach."""
import mpmath

from oracle.pointwise import PointOracle

mpmath.mp.dps = 40


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
