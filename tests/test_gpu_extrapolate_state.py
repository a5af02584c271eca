"""Parity of the other reading of Table B's extrapolation (config field
extrapolate_state = 1): at a stencil point outside the PE the state U is
extrapolated to level n with the weights w_l(k) and the differentiated
quantities are evaluated once from it, q(sum_l w_l U^{n-k-l}), instead of
sum_l w_l q(U^{n-k-l}).  The CUDA path (ghost kernel of every kernel path and
of the batch) against the oracle's rhs() with Config.extrapolate_state: the
FP64 form to 1e-12 per RHS and 1e-10 over 100 AT steps, the FP32 forms to
2e-4; each FP64 case is one where the two readings differ by far more than
the tolerance, so the flag is seen to act."""
import numpy as np
import pytest

from oracle import ns
from paper_2003_10561_gb300 import synth

pytestmark = pytest.mark.gpu

GAMMA, PR, OMEGA = 1.4, 0.7, 0.76


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2003_10561_gb300 import at_dns
    at_dns.load()
    return at_dns


def rel_linf(a, b):
    return [float(np.max(np.abs(a[v] - b[v])) / max(np.max(np.abs(b[v])), 1e-300)) for v in range(5)]


def make(lib, n, pes, precision="p64", path="auto", **kw):
    if path == "paired" and precision == "p64":
        pytest.skip("the paired kernel runs the FP32 forms only")
    try:
        return lib.Solver(n=n, pes=pes, precision=precision, path=path, extrapolate_state=1,
                          **{"gamma": GAMMA, "prandtl": PR, "visc_exp": OMEGA, **kw})
    except lib.AtDnsError as e:
        if path in ("fused", "paired") and e.code == lib.AT_DNS_E_UNSUPPORTED:
            pytest.skip("%s path does not apply to n=%s pes=%s" % (path, n, pes))
        raise


def ocfg(n, pes, xstate=True, **kw):
    return ns.Config(n=tuple(n), pes=tuple(pes), extrapolate_state=xstate,
                     **{"gamma": GAMMA, "prandtl": PR, "visc_exp": OMEGA, **kw})


CASES = [
    # n, pes, mode, step, L, order
    ((16, 16, 16), (2, 2, 2), "random", 9, 2, 4),
    ((16, 16, 16), (2, 2, 2), "periodic", 9, 2, 4),   # k = 1 on every face
    ((15, 12, 20), (3, 2, 4), "random", 11, 3, 4),      # ragged PEs, non-cubic
    ((24, 10, 16), (4, 1, 2), "random", 13, 4, 4),      # a direction without faces
    ((40, 24, 16), (5, 3, 2), "random", 10, 2, 4),      # 8^3 PEs (fused tiles)
    ((16, 16, 16), (2, 2, 2), "ordered", 11, 3, 4),
    ((28, 28, 28), (2, 2, 2), "random", 12, 2, 6),      # 6th order: T_l = 4 levels per delay
    ((32, 16, 16), (2, 2, 2), "random", 9, 2, 4),       # PEs 16 x 8 x 8 (paired tiles)
]


def _hist_and_delays(c, n, step, mode, lib):
    U0 = synth.initial_state(n, k0=3.0, mach_t=0.3, seed=11)
    hist = synth.history(U0, c.n_levels, eps=2e-2, seed=5)
    return hist, ns.delay_map(c, step, lib.MODES[mode])


@pytest.mark.parametrize("path", ["multipass", "fused"])
@pytest.mark.parametrize("n,pes,mode,step,L,order", CASES)
def test_rhs_parity_fp64(lib, n, pes, mode, step, L, order, path):
    kw = dict(mu0=0.02, dt=2e-3, max_delay=L, comm_period=L + 1, seed=77, order=order)
    c = ocfg(n, pes, **kw)
    hist, dm = _hist_and_delays(c, n, step, mode, lib)
    s = make(lib, n, pes, path=path, **kw)
    s.set_history(hist, step)
    R = s.rhs(mode)
    Rref = ns.rhs(c, hist, dm)
    err = rel_linf(R, Rref)
    assert max(err) <= 1e-12, err
    # the readings differ here by far more than the tolerance
    other = rel_linf(ns.rhs(ocfg(n, pes, xstate=False, **kw), hist, dm), Rref)
    assert max(other) > 1e-9, other


@pytest.mark.parametrize("prec", ["p32", "p32c"])
@pytest.mark.parametrize("path", ["multipass", "fused", "paired"])
@pytest.mark.parametrize("n,pes,mode,step,L,order", [CASES[0], CASES[2], CASES[4], CASES[5], CASES[7]])
def test_rhs_parity_fp32(lib, n, pes, mode, step, L, order, path, prec):
    kw = dict(mu0=0.02, dt=2e-3, max_delay=L, comm_period=L + 1, seed=77, order=order)
    c = ocfg(n, pes, **kw)
    hist, dm = _hist_and_delays(c, n, step, mode, lib)
    s = make(lib, n, pes, prec, path=path, **kw)
    s.set_history(hist, step)
    R = s.rhs(mode)
    err = rel_linf(R, ns.rhs(c, hist, dm))
    other = rel_linf(R, ns.rhs(ocfg(n, pes, xstate=False, **kw), hist, dm))
    print("fp32 %s %s n=%s %s: to this reading %s, to the other %s" % (prec, path, n, mode, err, other))
    assert max(err) <= 2e-4, err


@pytest.mark.parametrize("prec,path,tol", [("p64", "multipass", 1e-10), ("p64", "fused", 1e-10),
                                           ("p32c", "paired", 2e-4), ("p32", "fused", 2e-4)])
@pytest.mark.parametrize("mode", ["random", "ordered"])
def test_at_steps_parity(lib, mode, prec, path, tol):
    """2x2x2 PEs (of 16 x 8 x 8 points for the paired kernel, else 8^3), AT
    delays from the start-up on: 100 AB2 steps."""
    n, pes = ((32, 16, 16) if path == "paired" else (16, 16, 16)), (2, 2, 2)
    U0 = synth.initial_state(n, k0=3.0, mach_t=0.3, seed=21)
    kw = dict(mu0=0.03, dt=4e-3, max_delay=2, comm_period=3, seed=5)
    c = ocfg(n, pes, **kw)
    s = make(lib, n, pes, prec, path=path, **kw)
    s.set_state(U0)
    run = ns.Run.start(c, U0, lib.MODES[mode])
    for _ in range(100):
        run.step()
    s.step(100, mode)
    err = rel_linf(s.get_state(), run.levels[0])
    assert max(err) <= tol, err


def test_batch_member_keeps_its_reading(lib):
    """A batch of members with either reading: each ends bit-identical to the
    same member stepped alone."""
    base = dict(n=(16, 16, 16), pes=(2, 2, 2), mu0=0.02, dt=3e-3, max_delay=2, gamma=GAMMA, prandtl=PR,
                visc_exp=OMEGA)
    specs = [dict(base, precision="p64", seed=1, extrapolate_state=1),
             dict(base, precision="p64", seed=1, extrapolate_state=0),
             dict(base, precision="p32c", seed=2, extrapolate_state=1)]
    states = [synth.initial_state(sp["n"], k0=3.0, mach_t=0.2, seed=60 + i) for i, sp in enumerate(specs)]
    states[1] = states[0].copy()   # members 0 and 1 differ only in the reading
    batch = lib.Batch(specs)
    for m, U0 in zip(batch.members, states):
        m.set_state(U0)
    batch.step(12, "random")
    got = [m.get_state() for m in batch.members]
    for sp, g, U0 in zip(specs, got, states):
        alone = lib.Solver(**sp)
        alone.set_state(U0)
        alone.step(12, "random")
        assert np.array_equal(g, alone.get_state())
        alone.close()
    # same member, same start: the two readings part after the start-up
    assert not np.array_equal(got[0], got[1])
    batch.close()


def test_checkpoint_names_the_reading(lib):
    sp = dict(n=(16, 16, 16), pes=(2, 2, 2), precision="p64", mu0=0.02, dt=3e-3, max_delay=2, seed=3)
    a = make(lib, **sp)
    a.set_state(synth.initial_state(sp["n"], k0=3.0, mach_t=0.2, seed=4))
    a.step(3, "random")
    ck = a.checkpoint()
    other = lib.Solver(**sp)   # the default reading
    with pytest.raises(lib.AtDnsError) as e:
        other.restore(ck)
    assert "extrapolate_state" in str(e.value)
    other.close()
    a.close()
