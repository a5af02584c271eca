"""Full-size check of the memory-lean FP32-bulk configuration (the workload
list's fifth): 1024^3 with 16x16x16 virtual PEs of 64^3 (N_B = 17.6 %),
random AT delays with L = 4 (seven FP64 ring levels), forcing on
|kappa| <= 2, FP32 state and stencils with compensated FP32 accumulation and
FP64 reductions (P32C), on the paired fused path (no per-point work arrays).

The state is a smooth analytic, time-dependent field: the library receives it
as two device-resident levels (U^n and U^{n-1}; older ring levels repeat the
latter), and the pointwise oracle evaluates the same formula at sampled
points (no 1024^3 array ever reaches the host).  The RHS at step n, with that
step's random delay map and forcing, must match at the sampled points within
the FP32 tolerance scaled to this grid (2e-4 at 32^3, times 32 for the 1/dx
growth of the first-derivative stencil terms), and the handle must fit in
180 GB of device memory.  Then the run's 200 steps, timed, must stay healthy,
and are reported against the FP64 plain (synchronous, one PE) method on the
same analytic field at 512^3 on the same GPU.
"""
import math

import numpy as np
import pytest

from oracle import ns
from oracle.pointwise import PointOracle

pytestmark = pytest.mark.gpu

GAMMA, PR, OMEGA, MU0 = 1.4, 0.7, 0.76, 0.002
N, PES, L, STEP, DT = 1024, 16, 4, 20, 2e-4
TOL = 2e-4 * 32


def _prims(x, y, z, t, lib):
    s, c = lib.sin, lib.cos
    rho = 1 + 0.1 * s(x + 0.3 * t) * c(y) + 0.05 * s(z - 0.2 * t)
    u = 0.2 * s(y) * c(z + 0.1 * t) + 0.1 * c(x)
    v = 0.15 * s(z) * c(x - 0.2 * t) + 0.05 * s(y)
    w = 0.1 * s(x) * s(y + 0.3 * t) + 0.08 * c(z)
    T = 1 + 0.1 * c(x - y) * s(z + 0.2 * t)
    return rho, u, v, w, T


def _conserved(x, y, z, t, lib):
    rho, u, v, w, T = _prims(x, y, z, t, lib)
    E = rho * T / (GAMMA * (GAMMA - 1.0)) + 0.5 * rho * (u * u + v * v + w * w)
    return rho, rho * u, rho * v, rho * w, E


class AnalyticLevel:
    """Level l of the history (t = t_n - min(l, 1) dt), indexed [v, z, y, x]."""

    def __init__(self, l):
        self.t = -min(l, 1) * DT

    def __getitem__(self, key):
        v, z, y, x = key
        h = 2 * math.pi / N
        return _conserved(x * h, y * h, z * h, self.t, math)[v]


def test_config5_1024_fp32_bulk_memory_parity_and_200_steps():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    free, total = torch.cuda.mem_get_info()
    if free < 265e9:
        pytest.skip("needs about 265 GB of free device memory (the handle and two FP64 levels)")
    from paper_2003_10561_gb300 import at_dns
    kw = dict(gamma=GAMMA, prandtl=PR, visc_exp=OMEGA, mu0=MU0, dt=DT, max_delay=L, seed=97,
              forcing=1, kf=2.0, f_amp=0.02, f_tcorr=0.5, f_seed=13)
    stream = torch.cuda.Stream()
    s = at_dns.Solver(n=(N, N, N), pes=(PES, PES, PES), precision="p32c", path="paired", stream=stream.cuda_stream,
                      **kw)
    info = s.info()
    assert info["device_bytes"] <= 180e9, info["device_bytes"]
    assert info["tile"] == [32, 8, 64] and info["kernel_path"] == at_dns.AT_DNS_PATH_PAIRED

    # two levels on the device, filled plane block by plane block
    lv = torch.empty((2, 5, N, N, N), dtype=torch.float64, device="cuda")
    ax = torch.arange(N, dtype=torch.float64, device="cuda") * (2 * math.pi / N)
    X = ax.view(1, 1, N)
    Y = ax.view(1, N, 1)
    for l in range(2):
        t = -l * DT
        for z0 in range(0, N, 64):
            Z = ax[z0:z0 + 64].view(64, 1, 1)
            vals = _conserved(X, Y, Z, t, torch)
            for var in range(5):
                lv[l, var, z0:z0 + 64] = vals[var]
    torch.cuda.synchronize()   # the levels were built on torch's stream, the handle runs on its own
    s.set_history(lv, STEP)
    del lv, vals
    torch.cuda.empty_cache()
    R = torch.empty((5, N, N, N), dtype=torch.float64, device="cuda")
    s.rhs("random", R)
    torch.cuda.synchronize()

    cfg = ns.Config(n=(N, N, N), pes=(PES, PES, PES), **{**kw, "forcing": True})
    po = PointOracle(cfg, AnalyticLevel, ns.delay_map(cfg, STEP, ns.RANDOM), ns.forcing_coefficients(cfg, STEP),
                     ns.forcing_modes(cfg.kf))
    rng = np.random.default_rng(3)
    nl = N // PES
    pts = [tuple(int(v) for v in rng.integers(0, N, 3)) for _ in range(60)]
    for a in (0, 1, nl - 2, nl - 1, nl, nl + 1, 5 * nl + 3):
        pts.append((a, 7 * nl + 1, (a + 3) % N))
        pts.append((3 * nl + 2, a, 11 * nl))
        pts.append((N - 1, 5, a))
    ref = np.array([po.rhs(p) for p in pts])
    idx = torch.tensor([(z * N + y) * N + x for (x, y, z) in pts], device="cuda")
    got = torch.stack([R[v].reshape(-1)[idx] for v in range(5)], dim=1).cpu().numpy()
    err = np.max(np.abs(got - ref), axis=0) / np.max(np.abs(ref), axis=0)
    assert np.max(err) <= TOL, err

    # the configuration's 200 steps, timed, stay healthy
    del R
    torch.cuda.empty_cache()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    s.step(200, "random")
    e1.record(stream)
    torch.cuda.synchronize()
    rate32 = N ** 3 * 200 / (e0.elapsed_time(e1) / 1e3)
    st = s.stats()
    assert st["unstable"] == 0 and st["step"] == STEP + 199
    s.close()
    torch.cuda.empty_cache()

    # the FP64 plain method (synchronous, no PE faces) at 512^3 on the same field
    n2 = 512
    p = at_dns.Solver(n=(n2, n2, n2), pes=(1, 1, 1), precision="p64", stream=stream.cuda_stream,
                      **{**kw, "max_delay": 0})
    ax2 = torch.arange(n2, dtype=torch.float64, device="cuda") * (2 * math.pi / n2)
    U2 = torch.stack(_conserved(ax2.view(1, 1, n2), ax2.view(1, n2, 1), ax2.view(n2, 1, 1), 0.0, torch))
    U2 = U2.contiguous()
    torch.cuda.synchronize()
    p.set_state(U2)
    del U2
    p.step(3, "sync")
    torch.cuda.synchronize()
    e0.record(stream)
    p.step(20, "sync")
    e1.record(stream)
    torch.cuda.synchronize()
    rate64 = n2 ** 3 * 20 / (e0.elapsed_time(e1) / 1e3)
    assert p.stats()["unstable"] == 0
    p.close()
    print("config 5: 1024^3 FP32-bulk AT (L = 4) %.3e updates/s; 512^3 FP64 plain %.3e updates/s; ratio %.2f"
          % (rate32, rate64, rate32 / rate64))
    assert rate32 > rate64
