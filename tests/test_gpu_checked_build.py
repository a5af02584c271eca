"""The bounds-checked build: every translation unit compiled with
-DAT_DNS_CHECKS, so the index checks on the ring, ghost-array, state and
staging accesses of the ghost, ring-store and paired kernels are compiled
in (a failed check records its class in the device step state, redirects
the access to index 0 and makes the call return AT_DNS_E_BOUNDS).  In a
child process that loads libat_dns_checked.so, parity cases on every path
-- FP64 multi-pass with forcing, P32C paired, P32 fused, ragged PEs, the
6th order, AB2 steps on graph replay, a persistent batch and a checkpoint
round trip -- match the oracle with no failed check.  (This stands in for
a memory checker, which is not available on the GPU pool.)"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r'''
import numpy as np
import torch
from oracle import ns
from paper_2003_10561_gb300 import at_dns, synth
lib = at_dns.load()
assert lib._name.endswith("libat_dns_checked.so"), lib._name
kw = dict(gamma=1.4, prandtl=0.7, visc_exp=0.76, mu0=0.02, dt=2e-3, max_delay=2, seed=7)
cases = [
    ((16, 16, 16), (2, 2, 2), "p64", "multipass", 4, dict(forcing=1, kf=3.0, f_amp=0.05, f_tcorr=0.5, f_seed=3)),
    ((15, 12, 20), (3, 2, 4), "p64", "multipass", 4, {}),
    ((32, 32, 32), (2, 2, 2), "p32c", "paired", 4, {}),
    ((32, 32, 32), (2, 2, 2), "p32", "fused", 4, {}),
    ((32, 16, 16), (2, 1, 2), "p32c", "fused", 4, {}),
    ((14, 14, 14), (2, 2, 2), "p64", "multipass", 6, {}),
    ((28, 28, 28), (2, 2, 2), "p32c", "multipass", 6, {}),
]
st = torch.cuda.Stream()
for n, pes, prec, path, order, extra in cases:
    cfg_kw = dict(kw, order=order, **extra)
    cfg = ns.Config(n=n, pes=pes, **{**cfg_kw, "forcing": bool(extra.get("forcing", 0))})
    U0 = synth.initial_state(n, k0=3.0, mach_t=0.3, seed=1)
    hist = synth.history(U0, cfg.n_levels, eps=2e-2, seed=2)
    step = cfg.n_levels + 4
    s = at_dns.Solver(n=n, pes=pes, precision=prec, path=path, stream=st.cuda_stream, **cfg_kw)
    s.set_history(hist, step)
    R = s.rhs("random")
    fhat = ns.forcing_coefficients(cfg, step) if cfg.forcing else None
    ref = ns.rhs(cfg, hist, ns.delay_map(cfg, step, ns.RANDOM), fhat)
    err = max(float(np.max(np.abs(R[v] - ref[v])) / np.max(np.abs(ref[v]))) for v in range(5))
    tol = 1e-12 if prec == "p64" else (3e-4 if order == 6 else 2e-4)
    assert err <= tol, (n, pes, prec, path, order, err)
    s.step(6, "random")
    ck = s.checkpoint()
    s.restore(ck)
    s.step(2, "periodic")
    assert np.all(np.isfinite(s.get_state()))
    s.close()
spec = dict(n=(32, 32, 32), pes=(2, 2, 2), precision="p32c", stats_every=1, **kw)
b = at_dns.Batch([spec, dict(spec, n=(48, 48, 48), pes=(3, 3, 3), seed=8)], persistent=True)
assert b.persistent
for i, m in enumerate(b.members):
    m.set_state(synth.initial_state(m.n, k0=3.0, mach_t=0.2, seed=10 + i))
b.step(8, "random")
b.close()
print("checked ok", len(cases))
'''


def test_checked_build_runs_parity_cases_without_a_failed_check():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2003_10561_gb300 import build
    build.build(checked=True)
    env = dict(os.environ, AT_DNS_LIBRARY="checked")
    r = subprocess.run([sys.executable, "-c", SCRIPT], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=1200)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "checked ok 7" in r.stdout
