"""Stability limit of the Navier-Stokes solver under the fixed worst-case
delay (Sec. 3.2): bisection on the convective CFL for decaying turbulence
at 64^3 with 4x4x4 PEs of 16^3, L = 0 .. 3.  The limit must fall with L
(f(L) = r_c,max(0) / r_c,max(L) > 1 and growing), the trend the paper fits
with 0.90 L^2 - 0.35 L + 1."""
import pytest

from paper_2003_10561_gb300 import stability, synth

pytestmark = pytest.mark.gpu


def test_ns_cfl_limit_falls_with_delay():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2003_10561_gb300 import at_dns
    n = (64, 64, 64)
    mu0 = synth.mu0_for_resolution(n, k0=4.0, mach_t=0.3, seed=0)
    U0 = synth.initial_state(n, k0=4.0, mach_t=0.3, seed=0)
    stream = torch.cuda.Stream()
    limits = []
    for L in range(0, 4):
        def make(cfl, L=L):
            return at_dns.Solver(n=n, pes=(4, 4, 4), gamma=1.4, prandtl=0.7, visc_exp=0.76, mu0=mu0, cfl=cfl,
                                 dt=0.0, max_delay=max(L, 1), comm_period=1, stream=stream.cuda_stream,
                                 stats_every=0)
        limits.append(stability.ns_cfl_limit(make, U0, L, steps=300, lo=0.005))
    print("r_c,max(L) =", limits, "f(L) =", [limits[0] / x if x > 0 else None for x in limits])
    assert 0.2 < limits[0] < 2.0
    assert all(x > 0 for x in limits), limits
    for a, b in zip(limits, limits[1:]):
        assert b < a, limits
