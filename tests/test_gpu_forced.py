"""A forced stationary field made with the library's own forcing (the
stand-in for the paper's forced fields, Sec. 4.2): 32^3 from a weak initial
field, forcing on |kappa| <= 2, run in blocks until the block-mean kinetic
energy changes by less than 5 %; the field then has a finite positive
dissipation and its energy spectrum peaks at the forced scales."""
import numpy as np
import pytest

from paper_2003_10561_gb300 import analysis, synth

pytestmark = pytest.mark.gpu


def test_forced_run_reaches_stationarity():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2003_10561_gb300 import at_dns
    n = (32, 32, 32)
    mu0 = 0.05
    U0 = synth.initial_state(n, k0=2.0, mach_t=0.2, seed=7)
    stream = torch.cuda.Stream()
    s = at_dns.Solver(n=n, pes=(2, 2, 2), stream=stream.cuda_stream, mu0=mu0, cfl=0.2, dt=0.0, forcing=1,
                      kf=2.0, f_amp=0.005, f_tcorr=0.5, f_seed=3)
    U, hist = analysis.forced_stationary_state(s, U0, block=100, max_blocks=60, tol=0.05)
    s.close()
    assert len(hist) >= 2 and abs(hist[-1] - hist[-2]) <= 0.05 * hist[-2], hist
    a = analysis.analyze(U, mu0=mu0)
    assert a["eps"] > 0
    assert int(np.argmax(a["E"][1:])) + 1 <= 3, a["E"][:6]
