"""The allocation-free right-hand side (at_dns_rhs_noalloc) against the regular
entry point.

at_dns_rhs_noalloc exists for callers that cannot allocate device memory (a
host framework that owns every allocation, a region that must not allocate
or synchronise, a plugin in a process that forbids new allocations); its work
arrays live in a fixed file-scope device array shared by all calls.  This
test calls it through the C ABI twice in a row with different states (the
second call must not see the first one's leftovers), at a ragged size and at
the size limit, then a smaller grid right after the largest one with the
second call on a non-default stream, and compares each result with at_dns_rhs
of a one-PE synchronous handle.  Oversized problems and a non-finite
viscosity exponent must be rejected before any GPU work.
"""
import numpy as np
import pytest

from paper_2003_10561_gb300 import synth

pytestmark = pytest.mark.gpu

GAMMA, PR, MU0, OMEGA = 1.4, 0.7, 0.02, 0.76


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2003_10561_gb300 import at_dns
    at_dns.load()
    return torch, at_dns


def _state(n, seed):
    U0 = synth.initial_state(n, k0=3.0, mach_t=0.3, seed=seed, gamma=GAMMA)
    return synth.history(U0, 1, eps=2e-2, seed=seed + 1)[0]


def _reference(at_dns, n, U):
    s = at_dns.Solver(n=n, pes=(1, 1, 1), precision="p64", gamma=GAMMA, prandtl=PR, mu0=MU0,
                      visc_exp=OMEGA, dt=1e-3)
    s.set_state(U)
    R = s.rhs("sync")
    s.close()
    return R


def _rel_linf(a, b):
    return max(float(np.max(np.abs(a[v] - b[v])) / np.max(np.abs(b[v]))) for v in range(5))


@pytest.mark.parametrize("n", [(24, 20, 16), (64, 64, 64)])
def test_noalloc_rhs_matches_at_dns_rhs_twice(env, n):
    torch, at_dns = env
    for seed in (3, 8):                       # two calls in a row, different states
        U = _state(n, seed)
        u = torch.from_numpy(U).cuda()
        r = torch.full_like(u, float("nan"))
        at_dns.at_dns_rhs_noalloc(n, GAMMA, PR, MU0, OMEGA, u, r)
        torch.cuda.synchronize()
        got = r.cpu().numpy()
        ref = _reference(at_dns, n, U)
        assert np.all(np.isfinite(got))
        assert _rel_linf(got, ref) <= 1e-12


def test_noalloc_small_after_large_on_a_side_stream(env):
    """A smaller problem right after a larger one (the shared array still holds
    the larger call's work arrays), the second call queued on a non-default
    stream whose handle is passed through the C ABI."""
    torch, at_dns = env
    side = torch.cuda.Stream()
    for n, stream in (((64, 64, 64), None), ((24, 20, 16), side)):
        U = _state(n, 11)
        u = torch.from_numpy(U).cuda()
        r = torch.full_like(u, float("nan"))
        torch.cuda.synchronize()
        if stream is None:
            at_dns.at_dns_rhs_noalloc(n, GAMMA, PR, MU0, OMEGA, u, r)
        else:
            with torch.cuda.stream(stream):
                at_dns.at_dns_rhs_noalloc(n, GAMMA, PR, MU0, OMEGA, u, r, stream=stream.cuda_stream)
        torch.cuda.synchronize()
        got = r.cpu().numpy()
        ref = _reference(at_dns, n, U)
        assert np.all(np.isfinite(got))
        assert _rel_linf(got, ref) <= 1e-12


def test_noalloc_rejects_non_finite_exponent(env):
    torch, at_dns = env
    n = (16, 16, 16)
    u = torch.ones(5 * 16 ** 3, dtype=torch.float64, device="cuda")
    r = torch.empty_like(u)
    for bad in (float("nan"), float("inf")):
        with pytest.raises(at_dns.AtDnsError) as ei:
            at_dns.at_dns_rhs_noalloc(n, GAMMA, PR, MU0, bad, u, r)
        assert ei.value.code == at_dns.AT_DNS_E_INVALID_ARG


def test_noalloc_rejects_oversized_problem(env):
    torch, at_dns = env
    n = (65, 64, 64)
    u = torch.ones(5 * 65 * 64 * 64, dtype=torch.float64, device="cuda")
    r = torch.empty_like(u)
    with pytest.raises(at_dns.AtDnsError) as ei:
        at_dns.at_dns_rhs_noalloc(n, GAMMA, PR, MU0, OMEGA, u, r)
    assert ei.value.code == at_dns.AT_DNS_E_TOO_LARGE
