"""Checkpoint and resume: the run state of a handle (U^n with its low words,
R^{n-1}, the FP64 slab ring, the forcing coefficients, the statistics record,
the step counter, the time step and the start-up flag) in one buffer.  The
delay map and the forcing noise are pure functions of (seed, step, PE, face)
and (f_seed, step, mode), so a handle of the same configuration that loads a
checkpoint continues the saved run bit for bit: through the start-up and
after it, with random AT delays, forced and decaying, in every precision form,
from host and device buffers, on graph replay, and when a handle rewinds to
its own checkpoint.  A checkpoint of another configuration is refused, naming
the field that differs."""
import numpy as np
import pytest

from paper_2003_10561_gb300 import synth

pytestmark = pytest.mark.gpu

STATS = ("tke", "dissipation", "enstrophy", "mass", "energy", "grad_m2", "forcing_power", "max_wave_speed")


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2003_10561_gb300 import at_dns
    at_dns.load()
    return at_dns


def _spec(precision, forcing, **kw):
    sp = dict(n=(32, 32, 32), pes=(2, 2, 2), precision=precision, gamma=1.4, prandtl=0.7, visc_exp=0.76, mu0=0.02,
              dt=2e-3, max_delay=2, seed=11, stats_every=1, forcing=forcing, kf=2.0, f_amp=0.05, f_tcorr=0.5,
              f_seed=5)
    sp.update(kw)
    return sp


@pytest.mark.parametrize("precision,forcing", [("p64", 0), ("p64", 1), ("p32c", 1), ("p32", 0)])
@pytest.mark.parametrize("at_step", [2, 9])
def test_resume_continues_bit_for_bit(lib, precision, forcing, at_step):
    """Checkpoint after 2 steps (inside the start-up of L + T_l = 5 synchronous
    steps) or after 9 (delays active); the run continued by a fresh handle
    from the checkpoint equals the uninterrupted run in every bit, and so do
    its statistics; the saving handle rewound to its checkpoint repeats it."""
    sp = _spec(precision, forcing)
    U0 = synth.initial_state(sp["n"], k0=3.0, mach_t=0.2, seed=21)
    a = lib.Solver(**sp)
    a.set_state(U0)
    a.step(at_step, "random")
    ck = a.checkpoint()
    a.step(7, "random")
    ua, sa = a.get_state(), a.stats()
    b = lib.Solver(**sp)
    b.restore(ck)
    assert b.info()["step"] == at_step
    b.step(7, "random")
    assert np.array_equal(b.get_state(), ua)
    sb = b.stats()
    assert sb["step"] == sa["step"]
    for k in STATS:
        assert sb[k] == sa[k], k
    a.restore(ck)
    a.step(7, "random")
    assert np.array_equal(a.get_state(), ua)
    a.close()
    b.close()


def test_resume_from_device_buffer_on_graph_replay(lib):
    """The checkpoint in a CUDA tensor, loaded by a handle on its own stream
    (steps replayed from a captured graph): the same bits as the saving run;
    the statistics record right after the load is the saved one."""
    import torch
    sp = _spec("p32c", 1)
    U0 = synth.initial_state(sp["n"], k0=3.0, mach_t=0.2, seed=22)
    st = torch.cuda.Stream()
    a = lib.Solver(stream=st.cuda_stream, **sp)
    a.set_state(U0)
    a.step(10, "random")
    s_at = a.stats()
    buf = torch.empty(lib.at_dns_checkpoint_size(a.h), dtype=torch.uint8, device="cuda")
    a.checkpoint(buf)
    a.step(6, "random")
    ua = a.get_state()
    b = lib.Solver(stream=st.cuda_stream, **sp)
    b.restore(buf)
    s_b = b.stats()
    for k in STATS:
        assert s_b[k] == s_at[k], k
    b.step(6, "random")
    assert np.array_equal(b.get_state(), ua)
    a.close()
    b.close()


def test_checkpoint_of_another_configuration_is_refused(lib):
    sp = _spec("p64", 0)
    a = lib.Solver(**sp)
    a.set_state(synth.initial_state(sp["n"], k0=3.0, mach_t=0.2, seed=23))
    a.step(3, "random")
    ck = a.checkpoint()
    for change, field in ((dict(seed=12), "seed"), (dict(pes=(2, 2, 1)), "pes"), (dict(mu0=0.03), "physical"),
                          (dict(precision="p32c"), "precision")):
        other = lib.Solver(**dict(_spec("p64", 0), **change))
        with pytest.raises(lib.AtDnsError) as e:
            other.restore(ck)
        assert field in str(e.value), (field, str(e.value))
        other.close()
    bad = np.zeros_like(ck)
    with pytest.raises(lib.AtDnsError):
        a.restore(bad)
    a.close()
