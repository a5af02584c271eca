"""Pins of the stability tooling (Sec. 3.2, Appendix A) against the values the
paper reports and against closed forms:

* order 2 + forward Euler, delay L on both faces: r_d,max(0) = 1/2 and
  f(L) = L + 1 (the paper's fit, here exact: r_d,max(L) = 1/(2(L+1)));
* the same with the delay on one face: r_d,max(1) = 0.33 and a linear
  f(L) with slope 0.56 (Appendix A);
* order 4 + AB2: r_d,max(0) = 3/16 (AB2's real stability interval [-1, 0]
  over the largest D2 eigenvalue 16/3) -- the paper's 0.18 -- and, with
  one-sided delays, f(L) within 15 % of the paper's fit 0.74 L^2 + 0.47 L + 1;
* the companion matrix of Sec. 3.2 has the spectral radius of the
  Z-transform roots at the line's discrete phases.
"""
import numpy as np
import pytest

from oracle import ns
from paper_2003_10561_gb300 import stability as st


def test_order2_two_sided_exact_f():
    assert abs(st.rd_max(0) - 0.5) < 2e-6
    for L in range(1, 5):
        assert abs(st.rd_max(L) * (L + 1) - 0.5) < 1e-5, L


def test_order2_one_sided_appendix_values():
    rds = [st.rd_max(L, one_sided=True) for L in range(0, 5)]
    assert abs(rds[1] - 0.33) < 0.005
    slope, icpt = st.fit_f(range(5), rds, 1)
    assert abs(slope - 0.56) < 0.05 and abs(icpt - 0.9) < 0.1


def test_order4_ab2_limits():
    assert abs(st.rd_max(0, order=4) - 3.0 / 16.0) < 2e-6
    for L in range(1, 5):
        f = st.rd_max(0, order=4) / st.rd_max(L, order=4, one_sided=True)
        paper = 0.74 * L * L + 0.47 * L + 1.0
        assert abs(f / paper - 1.0) < 0.15, (L, f, paper)
        # delays on both faces are stricter than on one
        assert st.rd_max(L, order=4) < st.rd_max(L, order=4, one_sided=True)


@pytest.mark.parametrize("L,rd", [(0, 0.4), (1, 0.3), (2, 0.2), (2, 0.1)])
def test_companion_matrix_matches_z_transform(L, rd):
    N = 12
    rho = max(abs(np.linalg.eigvals(st.companion_matrix(N, L, rd))))
    rz = max(max(abs(st.roots(L, rd, 2 * np.pi * j / N))) for j in range(N))
    assert abs(rho - rz) < 1e-9


def test_fixed_delay_map():
    cfg = ns.Config(n=(16, 16, 16), pes=(2, 2, 2), max_delay=3)
    assert not ns.delay_map(cfg, cfg.n_levels - 1, ns.FIXED).any()
    assert (ns.delay_map(cfg, cfg.n_levels, ns.FIXED) == 3).all()


class _FakeSolver:
    """Stands in for a library handle: a run is stable when its CFL is at most
    `limit`; above it the kinetic energy grows, or (far above) the library
    reports an unstable state."""

    def __init__(self, cfl, limit, log):
        self.cfl, self.limit, self.log = cfl, limit, log
        self.k = 1.0

    def set_state(self, state):
        self.k = 1.0

    def stats(self):
        return {"tke": self.k}

    def step(self, n, mode):
        self.log.append(mode)
        if self.cfl > 2.0 * self.limit:
            from paper_2003_10561_gb300 import at_dns
            raise at_dns.AtDnsError(at_dns.AT_DNS_E_UNSTABLE, "non-finite")
        if self.cfl > self.limit:
            self.k *= 10.0

    def close(self):
        pass


@pytest.mark.parametrize("limit", [0.07, 0.2, 0.55])
def test_ns_cfl_limit_bisects_to_the_threshold(limit):
    """The bisection brackets the stability threshold within its tolerance,
    runs the fixed worst-case delay for L > 0 (sync for L = 0), and treats
    the library's unstable-state error as instability."""
    log = []
    got = st.ns_cfl_limit(lambda cfl: _FakeSolver(cfl, limit, log), None, L=2, lo=0.05, hi=2.0, tol=0.01)
    assert limit - 0.01 <= got <= limit
    assert set(log) == {"fixed"}
    log.clear()
    st.ns_cfl_limit(lambda cfl: _FakeSolver(cfl, limit, log), None, L=0, lo=0.05, hi=2.0, tol=0.01)
    assert set(log) == {"sync"}


def test_ns_cfl_limit_zero_when_even_the_lower_bound_fails():
    assert st.ns_cfl_limit(lambda cfl: _FakeSolver(cfl, 0.01, []), None, L=1, lo=0.05) == 0.0
