"""GPU parity: the CUDA library (through its C ABI) against the FP64 oracle.

Inputs come only from the seeded generator (paper_2003_10561_gb300.synth);
every expected value is computed by oracle/.  Tolerances:
* delay maps: bit-exact;
* FP64 form: relative L-infinity per conserved variable <= 1e-12 for one RHS,
  <= 1e-10 after 100 AB2 steps;
* FP32-bulk form: relative L-infinity per RHS <= 2e-4 (derived in the design
  notes from FP32 rounding of the 4th-order stencils: eps_32 times the
  cancellation factor of the second-derivative stencil at these grids).
"""
import math

import numpy as np
import pytest

from oracle import ns
from oracle.pointwise import PointOracle
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


PATHS = ["multipass", "fused"]
PATHS32 = PATHS + ["paired"]   # the paired kernel runs the FP32 forms only


def make(lib, n, pes, precision="p64", path="auto", **kw):
    """A solver on the requested kernel path; skips when the fused (or paired)
    path does not apply to this grid / PE shape or precision."""
    if path == "paired" and precision == "p64":
        pytest.skip("the paired kernel runs the FP32 forms only")
    try:
        return lib.Solver(n=n, pes=pes, precision=precision, path=path, **{"gamma": GAMMA, "prandtl": PR,
                                                                          "visc_exp": OMEGA, **kw})
    except lib.AtDnsError as e:
        if path in ("fused", "paired") and e.code == lib.AT_DNS_E_UNSUPPORTED:
            pytest.skip("%s path does not apply to n=%s pes=%s" % (path, n, pes))
        raise


def ocfg(n, pes, **kw):
    return ns.Config(n=tuple(n), pes=tuple(pes), **{"gamma": GAMMA, "prandtl": PR, "visc_exp": OMEGA, **kw})


# --------------------------------------------------------------------------
@pytest.mark.parametrize("mode", ["sync", "periodic", "random", "fixed", "ordered"])
def test_delay_map_bit_exact(lib, mode):
    s = make(lib, (40, 30, 20), (4, 3, 2), mu0=0.01, dt=1e-3, max_delay=3, comm_period=4,
             seed=0x0123456789ABCDEF)
    c = ocfg((40, 30, 20), (4, 3, 2), max_delay=3, comm_period=4, seed=0x0123456789ABCDEF)
    m = lib.MODES[mode]
    for step in (0, 5, 6, 7, 11, 100, 12345, 2 ** 31 + 7):
        gpu = s.delay_map(step, mode)
        ref = ns.delay_map(c, step, m)
        assert np.array_equal(gpu.astype(np.int64), ref), (mode, step)


# --------------------------------------------------------------------------
CASES = [
    # n, pes, mode, step, L
    ((32, 32, 32), (1, 1, 1), "sync", 0, 2),
    ((16, 16, 16), (2, 2, 2), "random", 9, 2),
    ((16, 16, 16), (2, 2, 2), "periodic", 8, 2),
    ((15, 12, 20), (3, 2, 4), "random", 11, 3),       # ragged PEs (5, 6, 5), non-cubic
    ((24, 10, 16), (4, 1, 2), "random", 13, 4),       # a direction without faces
    ((40, 24, 16), (5, 3, 2), "random", 10, 2),       # 8^3 PEs (fused tiles 8 x 8)
    ((48, 32, 24), (3, 2, 3), "periodic", 9, 2),      # 16 x 16 x 8 PEs
    ((32, 16, 24), (1, 2, 3), "random", 12, 3),       # x without faces, periodic wrap in a tile
    ((16, 16, 16), (2, 2, 2), "fixed", 9, 2),         # the worst case of the stability scans
    ((16, 16, 16), (2, 2, 2), "ordered", 11, 3),      # ordered random delays (in-order arrivals)
    ((15, 12, 20), (3, 2, 4), "ordered", 12, 2),
]


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("n,pes,mode,step,L", CASES)
def test_rhs_parity_fp64(lib, n, pes, mode, step, L, path):
    mu0 = 0.02
    U0 = synth.initial_state(n, k0=3.0, mach_t=0.3, seed=11)
    c = ocfg(n, pes, mu0=mu0, dt=2e-3, max_delay=L, comm_period=L + 1, seed=77)
    hist = synth.history(U0, c.n_levels, eps=2e-2, seed=5)
    s = make(lib, n, pes, path=path, mu0=mu0, dt=2e-3, max_delay=L, comm_period=L + 1, seed=77)
    s.set_history(hist, step)
    R = s.rhs(mode)
    Rref = ns.rhs(c, hist, ns.delay_map(c, step, lib.MODES[mode]))
    err = rel_linf(R, Rref)
    assert max(err) <= 1e-12, err


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("kf", [2.0, 3.0])
def test_rhs_parity_fp64_forced(lib, path, kf):
    """Forcing on the shell |kappa| <= kappa_f: 2 (the workload's, 16 modes in
    the half set) and 3 (the paper's, Sec. 4.2: 61 modes and wider x-line
    tables)."""
    n, pes = (16, 16, 16), (2, 2, 2)
    kw = dict(mu0=0.02, dt=5e-3, max_delay=2, seed=3, forcing=1, kf=kf, f_amp=0.2, f_tcorr=0.3, f_seed=99)
    U0 = synth.initial_state(n, k0=3.0, mach_t=0.3, seed=12)
    c = ocfg(n, pes, **{**kw, "forcing": True})
    assert len(ns.forcing_modes(kf)) == {2.0: 16, 3.0: 61}[kf]
    hist = synth.history(U0, c.n_levels, eps=1e-2, seed=6)
    s = make(lib, n, pes, path=path, **kw)
    s.set_history(hist, 9)
    R = s.rhs("random")
    Rref = ns.rhs(c, hist, ns.delay_map(c, 9, ns.RANDOM), ns.forcing_coefficients(c, 9))
    err = rel_linf(R, Rref)
    print("forced kf=%g %s fp64 rel err" % (kf, path), err)
    assert max(err) <= 1e-12, err


@pytest.mark.parametrize("path", PATHS32)
def test_rhs_parity_fp32_forced_kf3(lib, path):
    """The FP32-bulk form (compensated update, FP64 ring) with the paper's
    forcing shell kappa_f = 3 and random delays."""
    n, pes = (16, 16, 16), (2, 2, 2)
    kw = dict(mu0=0.02, dt=5e-3, max_delay=2, seed=3, forcing=1, kf=3.0, f_amp=0.2, f_tcorr=0.3, f_seed=99)
    U0 = synth.initial_state(n, k0=3.0, mach_t=0.3, seed=12)
    c = ocfg(n, pes, **{**kw, "forcing": True})
    hist = synth.history(U0, c.n_levels, eps=1e-2, seed=6)
    s = make(lib, n, pes, "p32c", path=path, **kw)
    s.set_history(hist, 9)
    R = s.rhs("random")
    Rref = ns.rhs(c, hist, ns.delay_map(c, 9, ns.RANDOM), ns.forcing_coefficients(c, 9))
    err = rel_linf(R, Rref)
    print("forced kf=3 %s p32c rel err" % path, err)
    assert max(err) <= 2e-4, err


@pytest.mark.parametrize("path", PATHS)
def test_stats_parity_fp64(lib, path):
    n, pes = (32, 32, 32), (2, 2, 2)
    U0 = synth.initial_state(n, k0=4.0, mach_t=0.3, seed=13)
    c = ocfg(n, pes, mu0=0.02, dt=1e-3, max_delay=2, seed=1)
    hist = synth.history(U0, c.n_levels, eps=1e-2, seed=2)
    s = make(lib, n, pes, path=path, mu0=0.02, dt=1e-3, max_delay=2, seed=1)
    s.set_history(hist, 9)
    s.rhs("random")
    st = s.stats()
    R, aux = ns.rhs(c, hist, ns.delay_map(c, 9, ns.RANDOM), None, True)
    ref = ns.statistics(c, hist[0], aux)
    for k, v in ref.items():
        g = st[k]
        if k == "mom":
            for a, b in zip(g, v):
                assert abs(a - b) <= 1e-12 * (abs(b) + 1e-3)
            continue
        assert abs(g - v) <= 1e-11 * abs(v) + 1e-15, (k, g, v)
    assert st["unstable"] == 0
    assert st["step"] == 9


@pytest.mark.parametrize("path", PATHS)
def test_config1_steps_parity_fp64(lib, path):
    """32^3, one PE, synchronous, CFL 0.5: 20 steps, then 100 (<= 1e-10)."""
    n = (32, 32, 32)
    mu0 = synth.mu0_for_resolution(n, k0=4.0, mach_t=0.3, seed=0)
    U0 = synth.initial_state(n, k0=4.0, mach_t=0.3, seed=0)
    c = ocfg(n, (1, 1, 1), mu0=mu0)
    c.dt = ns.dt_from_cfl(c, U0, 0.5)
    s = make(lib, n, (1, 1, 1), path=path, mu0=mu0, cfl=0.5, dt=0.0)
    s.set_state(U0)
    assert abs(s.info()["dt"] - c.dt) <= 1e-15 * c.dt
    run = ns.Run.start(c, U0, ns.SYNC)
    for k in range(100):
        run.step()
        if k + 1 in (20, 100):
            s.step(20 if k + 1 == 20 else 80, "sync")
            err = rel_linf(s.get_state(), run.levels[0])
            assert max(err) <= (1e-12 if k + 1 == 20 else 1e-10), (k + 1, err)


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("mode", ["random", "periodic", "ordered"])
def test_at_steps_parity_fp64(lib, mode, path):
    """16^3, 2x2x2 PEs, AT delays from the start-up on: 100 AB2 steps."""
    n, pes = (16, 16, 16), (2, 2, 2)
    U0 = synth.initial_state(n, k0=3.0, mach_t=0.3, seed=21)
    kw = dict(mu0=0.03, dt=4e-3, max_delay=2, comm_period=3, seed=5)
    c = ocfg(n, pes, **kw)
    s = make(lib, n, pes, path=path, **kw)
    s.set_state(U0)
    run = ns.Run.start(c, U0, lib.MODES[mode])
    for _ in range(100):
        run.step()
    s.step(100, mode)
    err = rel_linf(s.get_state(), run.levels[0])
    assert max(err) <= 1e-10, err


def test_zero_delay_equals_sync_fp64(lib):
    """Periodic mode during start-up and sync mode give bit-identical steps."""
    n, pes = (16, 16, 16), (2, 2, 2)
    U0 = synth.initial_state(n, seed=3)
    a = make(lib, n, pes, mu0=0.02, dt=3e-3, max_delay=2)
    b = make(lib, n, pes, mu0=0.02, dt=3e-3, max_delay=2)
    a.set_state(U0)
    b.set_state(U0)
    a.step(4, "random")    # steps 0..3 < L + 3: zero delays
    b.step(4, "sync")
    assert np.array_equal(a.get_state(), b.get_state())


# --------------------------------------------------------------------------
@pytest.mark.parametrize("prec", ["p32", "p32c"])
@pytest.mark.parametrize("path", PATHS32)
@pytest.mark.parametrize("n,pes,mode,step,L", CASES[:3] + CASES[5:7] + CASES[-2:-1])
def test_rhs_parity_fp32(lib, n, pes, mode, step, L, path, prec):
    U0 = synth.initial_state(n, k0=3.0, mach_t=0.3, seed=11)
    c = ocfg(n, pes, mu0=0.02, dt=2e-3, max_delay=L, comm_period=L + 1, seed=77)
    hist = synth.history(U0, c.n_levels, eps=2e-2, seed=5)
    s = make(lib, n, pes, prec, path=path, mu0=0.02, dt=2e-3, max_delay=L, comm_period=L + 1, seed=77)
    s.set_history(hist, step)
    R = s.rhs(mode)
    Rref = ns.rhs(c, hist, ns.delay_map(c, step, lib.MODES[mode]))
    err = rel_linf(R, Rref)
    print("fp32 %s %s n=%s pes=%s %s rel err" % (prec, path, n, pes, mode), err)
    assert max(err) <= 2e-4, err


# --------------------------------------------------------------------------


_EXT_CACHE = {}


def _extended_reference(c, hist, delays, pts):
    """The 40-digit right-hand side at the sampled points, from this machine's
    inputs (the inputs themselves differ between CPU architectures in their
    last bits, which moves the right-hand side by as much as the floor)."""
    ext_mod = pytest.importorskip("tests.extended")
    if "ext" not in _EXT_CACHE:
        pe = ext_mod.ExtendedPointOracle(c, lambda l: hist[l], delays)
        _EXT_CACHE["ext"] = np.array([[float(v) for v in pe.rhs(p)] for p in pts])
    return _EXT_CACHE["ext"]


# Tolerance at 256^3.  The FP64 bound is set by measurement: the FP64
# oracle's own rounding at these points, against a 40-digit evaluation of the
# same sums from the same inputs, is about 1.6e-12 of the scale of R_rho and
# 1.2e-12 of R_E (stencil terms of 1/dx times the field cancel to a small
# divergence), 1e-13 for the momenta.  The CUDA path evaluates the same sums
# in another order, so its error against the 40-digit values is bounded by
# four times that measured floor, or by 1e-12 where the floor allows.  The
# FP32 forms keep 2e-3: FP32 rounding times the same cancellation, scaled by
# the 8x of 1/dx from the 32^3 bound of 2e-4.
@pytest.mark.parametrize("path", PATHS32)
@pytest.mark.parametrize("precision,tol", [("p64", None), ("p32", 2e-3), ("p32c", 2e-3)])
def test_full_size_sampled_parity(lib, precision, tol, path):
    """256^3 with 8x8x8 PEs (the benchmark workload), random delays with L = 2,
    at a step past the start-up: sampled points against the brute-force
    pointwise oracle and against its 40-digit evaluation."""
    from tests.sampling import FULL_KW, FULL_N, FULL_PES, FULL_STEP, full_size_history, full_size_points
    if path == "paired" and precision == "p64":
        pytest.skip("the paired kernel runs the FP32 forms only")
    c, hist = full_size_history()
    s = make(lib, FULL_N, FULL_PES, precision, path=path, **FULL_KW)
    s.set_history(hist, FULL_STEP)
    R = s.rhs("random")
    s.close()
    delays = ns.delay_map(c, FULL_STEP, ns.RANDOM)
    po = PointOracle(c, lambda l: hist[l], delays)
    pts = full_size_points()
    ref = np.array([po.rhs(p) for p in pts])
    got = np.array([[R[v, z, y, x] for v in range(5)] for (x, y, z) in pts])
    xr = _extended_reference(c, hist, delays, pts)
    scale = np.max(np.abs(xr), axis=0)
    floor = np.max(np.abs(ref - xr), axis=0) / scale
    err_oracle = np.max(np.abs(got - ref), axis=0) / scale
    err_ext = np.max(np.abs(got - xr), axis=0) / scale
    print("256^3 sampled %s %s: rel err vs FP64 oracle" % (precision, path), err_oracle, "vs 40-digit", err_ext,
          "FP64 oracle floor", floor)
    if tol is None:
        bound = np.maximum(1e-12, 4.0 * floor)
        assert np.all(err_ext <= bound), (err_ext, bound)
    else:
        assert np.max(err_ext) <= tol and np.max(err_oracle) <= tol, (err_ext, err_oracle)


def test_unstable_state_reported(lib):
    """A state with negative density is reported as AT_DNS_E_UNSTABLE (host-made failure)."""
    n = (16, 16, 16)
    U0 = synth.initial_state(n, seed=2)
    U0[0, 3, 4, 5] = -1.0
    s = make(lib, n, (1, 1, 1), mu0=0.01, dt=1e-3)
    s.set_state(U0)
    with pytest.raises(lib.AtDnsError) as ei:
        s.step(2, "sync")
    assert ei.value.code == lib.AT_DNS_E_UNSTABLE
    st = s.stats()
    assert st["unstable"] != 0


def test_device_pointers_and_zero_steps(lib):
    import torch
    n = (16, 16, 16)
    U0 = synth.initial_state(n, seed=8)
    s = make(lib, n, (2, 2, 2), mu0=0.01, dt=1e-3)
    s.set_state(torch.from_numpy(U0).cuda())
    s.step(0, "random")
    out = torch.empty(U0.shape, dtype=torch.float64, device="cuda")
    s.get_state(out)
    assert np.array_equal(out.cpu().numpy(), U0)
    r_dev = torch.empty(U0.shape, dtype=torch.float64, device="cuda")
    s.rhs("sync", r_dev)
    r_host = s.rhs("sync")
    assert np.array_equal(r_dev.cpu().numpy(), r_host)


def test_paths_agree_and_report(lib):
    """Both kernel paths give the same steps up to rounding, and report themselves."""
    n, pes = (32, 32, 32), (4, 4, 4)
    U0 = synth.initial_state(n, seed=31)
    kw = dict(mu0=0.02, dt=3e-3, max_delay=2, seed=9)
    a = make(lib, n, pes, path="multipass", **kw)
    b = make(lib, n, pes, path="fused", **kw)
    assert make(lib, n, pes, **kw).info()["kernel_path"] == lib.AT_DNS_PATH_MULTIPASS
    assert a.info()["kernel_path"] == lib.AT_DNS_PATH_MULTIPASS
    assert b.info()["kernel_path"] == lib.AT_DNS_PATH_FUSED and b.info()["tile"] == [8, 8, 8]
    for s in (a, b):
        s.set_state(U0)
        s.step(12, "random")
    err = rel_linf(b.get_state(), a.get_state())
    assert max(err) <= 1e-12, err


def test_compensated_state_round_trip(lib):
    """The compensated form keeps ~48 bits of the state (hi + lo words); the
    plain FP32 form keeps 24."""
    n = (16, 16, 16)
    U0 = synth.history(synth.initial_state(n, seed=5), 1, eps=3e-2, seed=6)[0]
    a = make(lib, n, (2, 2, 2), "p32c", mu0=0.01, dt=1e-3)
    b = make(lib, n, (2, 2, 2), "p32", mu0=0.01, dt=1e-3)
    a.set_state(U0)
    b.set_state(U0)
    ea = max(rel_linf(a.get_state(), U0))
    eb = max(rel_linf(b.get_state(), U0))
    assert ea < 1e-12 and 1e-9 < eb < 1e-6, (ea, eb)


@pytest.mark.parametrize("path", PATHS)
def test_compensated_accumulation_keeps_small_increments(lib, path):
    """A uniform flow driven by a tiny force: every AB2 increment of the
    momentum lies below the FP32 resolution of the state.  The plain FP32 form
    drops them; the compensated form (TwoSum into a low word) accumulates them
    like FP64 (Eq. (time_ab) with FP32 arithmetic)."""
    n = (16, 16, 16)
    U0 = np.zeros((5,) + n[::-1])
    U0[0] = 1.0
    U0[1] = 0.3                               # uniform rho u
    U0[4] = (1.0 / GAMMA) / (GAMMA - 1.0) + 0.5 * 0.3 ** 2
    kw = dict(mu0=0.01, dt=1e-2, forcing=1, kf=1.0, f_amp=2e-7, f_tcorr=1e6, f_seed=4)
    out = {}
    for prec in ("p64", "p32", "p32c"):
        s = make(lib, n, (1, 1, 1), prec, path=path, **kw)
        s.set_state(U0)
        s.step(400, "sync")
        out[prec] = s.get_state()[1] - U0[1]
    ref = out["p64"]
    scale = np.max(np.abs(ref))
    assert scale > 1e-6                       # the force did change the momentum
    err_c = np.max(np.abs(out["p32c"] - ref)) / scale
    err_p = np.max(np.abs(out["p32"] - ref)) / scale
    # compensated: tracks FP64 up to the FP32 rounding of the stencil terms
    # (p and rho u u of a nearly uniform flow); plain FP32: increments lost
    assert err_c < 0.05 and err_p > 0.5 and err_c < err_p / 10, (err_c, err_p)


@pytest.mark.parametrize("path", PATHS)
def test_graph_replay_matches_direct_launches(lib, path):
    """Steps replayed from a captured one-step graph (handle on its own stream)
    equal steps launched kernel by kernel (legacy stream), bit for bit, with
    random delays and forcing active."""
    import torch
    n, pes = (16, 16, 16), (2, 2, 2)
    U0 = synth.initial_state(n, k0=3.0, seed=40)
    kw = dict(mu0=0.02, dt=3e-3, max_delay=2, seed=11, forcing=1, kf=2.0, f_amp=0.05, f_tcorr=0.4, f_seed=5)
    stream = torch.cuda.Stream()
    a = make(lib, n, pes, path=path, stream=stream.cuda_stream, **kw)
    b = make(lib, n, pes, path=path, **kw)
    for s in (a, b):
        s.set_state(U0)
        s.step(9, "random")
        s.step(3, "periodic")
    a.synchronize()
    assert np.array_equal(a.get_state(), b.get_state())
    sa, sb = a.stats(), b.stats()
    assert sa["step"] == sb["step"] == 11
    assert sa["tke"] == sb["tke"] and sa["dissipation"] == sb["dissipation"]


def test_batch_of_uneven_members_matches_members_alone(lib):
    """One graph launch per step advances members of different grids, PE
    layouts and precisions; each ends bit-identical to the same member stepped
    alone (config 4's batched ensemble, with seeds and Mach numbers varied)."""
    specs = [
        dict(n=(16, 16, 16), pes=(2, 2, 2), precision="p64", mu0=0.02, dt=3e-3, max_delay=2, seed=1),
        dict(n=(24, 24, 24), pes=(1, 1, 1), precision="p64", mu0=0.01, dt=2e-3, max_delay=2, seed=2),
        dict(n=(32, 32, 32), pes=(4, 4, 4), precision="p32", mu0=0.02, dt=2e-3, max_delay=2, seed=3),
        dict(n=(16, 24, 32), pes=(2, 3, 4), precision="p64", mu0=0.02, dt=2e-3, max_delay=2, seed=4,
             path="fused"),
    ]
    for sp in specs:
        sp.update(gamma=GAMMA, prandtl=PR, visc_exp=OMEGA)
    states = [synth.initial_state(sp["n"], k0=3.0, mach_t=0.1 + 0.1 * i, seed=50 + i) for i, sp in enumerate(specs)]
    batch = lib.Batch(specs)
    for m, U0 in zip(batch.members, states):
        m.set_state(U0)
    batch.step(8, "random")
    batch.step(4, "random")
    for sp, m, U0 in zip(specs, batch.members, states):
        alone = lib.Solver(**sp)
        alone.set_state(U0)
        alone.step(12, "random")
        assert np.array_equal(m.get_state(), alone.get_state())
        assert m.info()["step"] == 12
    batch.close()


def test_tuner_keeps_parity(lib):
    """The autotuner times every applicable kernel path / tile / z chunk and
    keeps the fastest; the result still matches the oracle."""
    n, pes, step = (32, 32, 32), (4, 4, 4), 9
    U0 = synth.initial_state(n, k0=3.0, seed=61)
    c = ocfg(n, pes, mu0=0.02, dt=2e-3, max_delay=2, seed=8)
    hist = synth.history(U0, c.n_levels, eps=2e-2, seed=62)
    s = make(lib, n, pes, mu0=0.02, dt=2e-3, max_delay=2, seed=8)
    s.set_history(hist, step)
    best = s.tune("random", trials=2)
    info = s.info()
    assert best > 0 and info["kernel_path"] in (lib.AT_DNS_PATH_MULTIPASS, lib.AT_DNS_PATH_FUSED)
    R = s.rhs("random")
    Rref = ns.rhs(c, hist, ns.delay_map(c, step, ns.RANDOM))
    assert max(rel_linf(R, Rref)) <= 1e-12


FUSED_SHAPES = [(32, 8), (16, 16), (16, 8), (8, 32), (8, 16), (8, 8), (32, 16)]


@pytest.mark.parametrize("prec", ["p64", "p32"])
def test_every_fused_tile_keeps_parity(lib, prec):
    """Each compiled fused tile shape and z chunk that applies (the autotuner's
    candidates), selected explicitly, matches the oracle."""
    n, pes = (64, 64, 32), (2, 2, 1)
    kw = dict(mu0=0.02, dt=2e-3, max_delay=2, seed=77)
    U0 = synth.initial_state(n, k0=3.0, mach_t=0.3, seed=11)
    c = ocfg(n, pes, **kw)
    hist = synth.history(U0, c.n_levels, eps=2e-2, seed=5)
    Rref = ns.rhs(c, hist, ns.delay_map(c, 9, ns.RANDOM))
    s = make(lib, n, pes, prec, **kw)
    s.set_history(hist, 9)
    tried = 0
    for tx, ty in FUSED_SHAPES:
        for zc in (32, 16, 8):
            try:
                s.set_kernel_path("fused", (tx, ty, zc))
            except lib.AtDnsError as e:
                assert e.code == lib.AT_DNS_E_UNSUPPORTED
                continue
            tried += 1
            R = s.rhs("random")
            err = rel_linf(R, Rref)
            assert max(err) <= (1e-12 if prec == "p64" else 2e-4), (tx, ty, zc, err)
    assert tried >= (18 if prec == "p64" else 21)


PAIRED_SHAPES = [(32, 8), (32, 16), (16, 16), (16, 8)]


@pytest.mark.parametrize("prec", ["p32", "p32c"])
def test_every_paired_tile_keeps_parity(lib, prec):
    """Each paired tile shape and z chunk (two points per thread, packed FP32
    arithmetic), selected explicitly, matches the oracle with random delays;
    a grid direction without PE faces (z) is covered too."""
    n, pes = (64, 64, 32), (2, 2, 1)
    kw = dict(mu0=0.02, dt=2e-3, max_delay=2, seed=77)
    U0 = synth.initial_state(n, k0=3.0, mach_t=0.3, seed=11)
    c = ocfg(n, pes, **kw)
    hist = synth.history(U0, c.n_levels, eps=2e-2, seed=5)
    Rref = ns.rhs(c, hist, ns.delay_map(c, 9, ns.RANDOM))
    s = make(lib, n, pes, prec, **kw)
    s.set_history(hist, 9)
    tried = 0
    for tx, ty in PAIRED_SHAPES:
        for zc in (32, 16, 8):
            s.set_kernel_path("paired", (tx, ty, zc))
            assert s.info()["kernel_path"] == lib.AT_DNS_PATH_PAIRED
            tried += 1
            R = s.rhs("random")
            err = rel_linf(R, Rref)
            print("paired %s tile %dx%dx%d rel err" % (prec, tx, ty, zc), err)
            assert max(err) <= 2e-4, (tx, ty, zc, err)
    assert tried == 12
    with pytest.raises(lib.AtDnsError) as ei:
        s.set_kernel_path("paired", (8, 8, 8))
    assert ei.value.code == lib.AT_DNS_E_UNSUPPORTED


def test_paired_graph_replay_matches_direct_launches(lib):
    """The paired kernel: graph-replayed steps equal kernel-by-kernel steps
    bit for bit (compensated form, random and periodic delays, forcing)."""
    import torch
    n, pes = (32, 32, 32), (2, 2, 2)
    U0 = synth.initial_state(n, k0=3.0, seed=40)
    kw = dict(mu0=0.02, dt=3e-3, max_delay=2, seed=11, forcing=1, kf=2.0, f_amp=0.05, f_tcorr=0.4, f_seed=5)
    stream = torch.cuda.Stream()
    a = make(lib, n, pes, "p32c", path="paired", stream=stream.cuda_stream, **kw)
    b = make(lib, n, pes, "p32c", path="paired", **kw)
    for s in (a, b):
        s.set_state(U0)
        s.step(9, "random")
        s.step(3, "periodic")
    a.synchronize()
    assert np.array_equal(a.get_state(), b.get_state())
    assert a.stats()["tke"] == b.stats()["tke"]


@pytest.mark.parametrize("prec", ["p32", "p32c"])
def test_paired_agrees_with_fused_and_fp64_over_steps(lib, prec):
    """30 AB2 steps with random delays and forcing from one state on the
    paired and the one-point-per-thread fused kernel (same arithmetic in a
    different instruction order) and in FP64: the two FP32 kernels agree to
    FP32 rounding, and both stay within the FP32 bound of the FP64 run."""
    n, pes = (32, 32, 32), (2, 2, 2)
    U0 = synth.initial_state(n, k0=3.0, mach_t=0.3, seed=44)
    kw = dict(mu0=0.02, dt=2e-3, max_delay=2, seed=12, forcing=1, kf=2.0, f_amp=0.1, f_tcorr=0.5, f_seed=6)
    out = {}
    for key, pr, path in (("p64", "p64", "multipass"), ("fused", prec, "fused"), ("paired", prec, "paired")):
        s = make(lib, n, pes, pr, path=path, **kw)
        s.set_state(U0)
        s.step(30, "random")
        out[key] = (s.get_state(), s.stats())
        s.close()
    d = max(rel_linf(out["paired"][0], out["fused"][0]))
    e_p = max(rel_linf(out["paired"][0], out["p64"][0]))
    e_f = max(rel_linf(out["fused"][0], out["p64"][0]))
    print("paired vs fused %.3e, paired vs fp64 %.3e, fused vs fp64 %.3e" % (d, e_p, e_f))
    assert d <= 1e-5 and e_p <= 2e-4 and e_f <= 2e-4
    for k in ("tke", "dissipation", "enstrophy"):
        ref = out["p64"][1][k]
        assert abs(out["paired"][1][k] - ref) <= 1e-4 * abs(ref), k


@pytest.mark.parametrize("prec,tol", [("p64", 1e-10), ("p32", 2e-4), ("p32c", 2e-4)])
@pytest.mark.parametrize("path", PATHS32)
def test_rk3_steps_parity(lib, path, prec, tol):
    """20 synchronous low-storage RK3 steps on 16^3 with 2x2x2 PEs (forced),
    through a captured graph on a stream, against the oracle's RK3."""
    torch = pytest.importorskip("torch")
    n, pes = (16, 16, 16), (2, 2, 2)
    kw = dict(mu0=0.03, dt=4e-3, max_delay=2, forcing=1, kf=2.0, f_amp=0.2, f_tcorr=0.3, f_seed=8)
    U0 = synth.initial_state(n, k0=3.0, mach_t=0.3, seed=21)
    c = ocfg(n, pes, **{**kw, "forcing": True}, integrator=ns.RK3)
    stream = torch.cuda.Stream()
    s = make(lib, n, pes, prec, path=path, stream=stream.cuda_stream, integrator=lib.AT_DNS_RK3, **kw)
    s.set_state(U0)
    run = ns.Run.start(c, U0, ns.SYNC)
    for _ in range(20):
        run.step()
    s.step(20, "sync")
    assert max(rel_linf(s.get_state(), run.levels[0])) <= tol
    with pytest.raises(lib.AtDnsError) as ei:
        s.step(1, "random")
    assert ei.value.code == lib.AT_DNS_E_UNSUPPORTED


def test_device_pool_from_a_tensor(lib):
    """All device buffers carved from a caller's tensor: the same steps as a
    handle that allocates its own memory, and OOM when the pool is too small."""
    torch = pytest.importorskip("torch")
    n, pes = (32, 32, 32), (2, 2, 2)
    kw = dict(mu0=0.02, dt=3e-3, max_delay=2, seed=4)
    U0 = synth.initial_state(n, k0=3.0, mach_t=0.3, seed=8)
    ref = make(lib, n, pes, **kw)
    need = ref.info()["device_bytes"] + 5 * n[0] * n[1] * n[2] * 8 + (1 << 16)   # + host staging
    pool = torch.empty(need + 4096, dtype=torch.uint8, device="cuda")
    s = make(lib, n, pes, pool=pool, **kw)
    for h in (ref, s):
        h.set_state(U0)
        h.step(10, "random")
    assert np.array_equal(s.get_state(), ref.get_state())
    assert s.info()["device_bytes"] <= pool.numel()
    assert np.array_equal(s.delay_map(12, "random"), ref.delay_map(12, "random"))
    s.close()
    small = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    with pytest.raises(lib.AtDnsError) as ei:
        make(lib, n, pes, pool=small, **kw)
    assert ei.value.code == lib.AT_DNS_E_OOM


def _fp32_ensemble_specs():
    """Uneven FP32 members whose PE extents are 16 (so each member alone takes
    the paired 16x16 tile, the persistent step's tile): both FP32 forms,
    different grids, PE counts, Mach numbers, viscosities and delay seeds."""
    specs = [
        dict(n=(32, 32, 32), pes=(2, 2, 2), precision="p32c", mu0=0.02, seed=1),
        dict(n=(48, 48, 48), pes=(3, 3, 3), precision="p32", mu0=0.015, seed=2),
        dict(n=(64, 32, 48), pes=(4, 2, 3), precision="p32c", mu0=0.01, seed=3),
        dict(n=(96, 96, 96), pes=(6, 6, 6), precision="p32c", mu0=0.008, seed=4),
        dict(n=(16, 16, 32), pes=(1, 1, 2), precision="p32", mu0=0.02, seed=5),
    ]
    for sp in specs:
        sp.update(gamma=GAMMA, prandtl=PR, visc_exp=OMEGA, dt=2e-3, max_delay=2, stats_every=1)
    states = [synth.initial_state(sp["n"], k0=3.0, mach_t=0.1 + 0.08 * i, seed=70 + i) for i, sp in enumerate(specs)]
    return specs, states


def _agree_below_fp32(a, b):
    """Largest difference per variable relative to the field's scale."""
    scale = np.max(np.abs(b.reshape(5, -1)), axis=1)
    return np.max(np.abs((a - b).reshape(5, -1)), axis=1) / scale


# Agreement of the persistent step with the kernels of a member stepped
# alone (the same operations compiled into another kernel, which may round
# single operations of the right-hand side differently; over the 12 steps of
# these tests the compensated form stayed within 1.3e-8 of each field's
# scale): 8 FP32 ulps of the scale (2^-20) for both FP32 forms.
PERSISTENT_BOUND = {"p32c": 2.0 ** -20, "p32": 2.0 ** -20}


def test_persistent_batch_matches_members_alone(lib):
    """The batched ensemble as one persistent kernel launch per step (ghost
    items and paired-kernel tiles of every member, each tile after its
    member's ghost items): every member agrees with the same member stepped
    alone on the paired 16x16 tile, through the start-up and with random
    delays, within PERSISTENT_BOUND, and its statistics within 1e-7.  The
    persistent step is deterministic: repeated runs, and identical members
    within one run, give identical bits."""
    specs, states = _fp32_ensemble_specs()
    runs = []
    for rep in range(2):
        batch = lib.Batch(specs, persistent=True)
        assert batch.persistent
        for m, U0 in zip(batch.members, states):
            m.set_state(U0)
        batch.step(7, "random")
        batch.step(5, "random")
        runs.append([m.get_state() for m in batch.members])
        stats = [m.stats() for m in batch.members]
        assert all(m.info()["step"] == 12 for m in batch.members)
        batch.close()
    for a, b in zip(*runs):
        assert np.array_equal(a, b)
    for sp, got, st, U0 in zip(specs, runs[0], stats, states):
        alone = lib.Solver(**sp)
        assert alone.info()["kernel_path"] == lib.AT_DNS_PATH_PAIRED and alone.info()["tile"][:2] == [16, 16]
        alone.set_state(U0)
        alone.step(12, "random")
        ref = alone.get_state()
        err = _agree_below_fp32(got, ref)
        assert np.all(err <= PERSISTENT_BOUND[sp["precision"]]), (sp, err)
        b = alone.stats()
        assert st["step"] == b["step"] == 11
        for k in ("tke", "dissipation", "enstrophy", "mass", "energy"):
            assert abs(st[k] - b[k]) <= 1e-7 * abs(b[k]), (k, st[k], b[k])
        alone.close()
    same = lib.Batch([specs[0]] * 4, persistent=True)
    for m in same.members:
        m.set_state(states[0])
    same.step(6, "random")
    outs = [m.get_state() for m in same.members]
    same.close()
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])


def test_persistent_batches_alternating_share_constant_memory(lib):
    """Two persistent batches stepped alternately (each step re-uploads the
    stepping batch's tile descriptions to constant memory, after the other
    batch's last launch) end bit-identical to each batch stepped on its own;
    a batch of 65 members (more descriptions than constant memory holds)
    takes the graph form."""
    specs, states = _fp32_ensemble_specs()
    groups = [(specs[:3], states[:3]), (specs[3:], states[3:])]

    def run(alternate):
        bs = [lib.Batch(sp, persistent=True) for sp, _ in groups]
        for b, (_, st) in zip(bs, groups):
            assert b.persistent
            for m, U0 in zip(b.members, st):
                m.set_state(U0)
        if alternate:
            for _ in range(4):
                for b in bs:
                    b.step(2, "random")
        else:
            for b in bs:
                b.step(8, "random")
        out = [[m.get_state() for m in b.members] for b in bs]
        for b in bs:
            b.close()
        return out

    for ga, gb in zip(run(True), run(False)):
        for a, b in zip(ga, gb):
            assert np.array_equal(a, b)
    many = lib.Batch([dict(specs[4], seed=100 + i) for i in range(65)])
    assert not many.set_persistent(True)
    many.close()


def test_persistent_wait_gives_up_and_context_survives(lib):
    """The bounded wait of the persistent step (a tile waiting for its
    member's ghost items) run on a counter that nothing advances returns
    unsatisfied after its poll limit (2^20 polls, well under a second), and
    the context stays usable: a solver steps afterwards."""
    import time
    t0 = time.perf_counter()
    assert lib.at_dns_wait_selftest(20)
    assert time.perf_counter() - t0 < 30
    specs, states = _fp32_ensemble_specs()
    s = lib.Solver(**specs[0])
    s.set_state(states[0])
    s.step(2, "random")
    assert np.all(np.isfinite(s.get_state()))
    s.close()


def test_batch_tune_keeps_states_and_runs_the_paths_it_picks(lib):
    """The batch autotuner times whole batch steps but restores every member's
    run state (bit for bit, step counter included); afterwards each member
    runs the path it picked, and a member stepped alone on its pre-tune path
    and then on its tuned path gives the same bits as in the batch."""
    specs, states = _fp32_ensemble_specs()
    batch = lib.Batch(specs)
    for m, U0 in zip(batch.members, states):
        m.set_state(U0)
    batch.step(3, "random")
    before = [m.get_state() for m in batch.members]
    paths0 = [(m.info()["kernel_path"], m.info()["tile"]) for m in batch.members]
    batch.tune("random", trials=1)
    for m, u in zip(batch.members, before):
        assert np.array_equal(m.get_state(), u)
        assert m.info()["step"] == 3
    paths1 = [(m.info()["kernel_path"], m.info()["tile"]) for m in batch.members]
    batch.step(4, "random")
    for sp, m, U0, p0, p1 in zip(specs, batch.members, states, paths0, paths1):
        alone = lib.Solver(**sp)
        lib.at_dns_set_kernel_path(alone.h, p0[0], p0[1])
        alone.set_state(U0)
        alone.step(3, "random")
        lib.at_dns_set_kernel_path(alone.h, p1[0], p1[1])
        alone.step(4, "random")
        assert np.array_equal(alone.get_state(), m.get_state()), (sp, p0, p1)
        alone.close()
    batch.close()


def test_persistent_and_graph_batch_steps_agree(lib):
    """The same ensemble stepped with the persistent launch and with the graph
    of per-member branches agrees within PERSISTENT_BOUND (each member takes
    the same paired tile either way); a batch with an FP64 member cannot take
    the persistent step."""
    specs, states = _fp32_ensemble_specs()
    out = []
    for persistent in (True, False):
        batch = lib.Batch(specs)
        assert batch.set_persistent(persistent) == persistent
        for m, U0 in zip(batch.members, states):
            m.set_state(U0)
        batch.step(10, "periodic")
        out.append([m.get_state() for m in batch.members])
        batch.close()
    for sp, a, b in zip(specs, *out):
        err = _agree_below_fp32(a, b)
        assert np.all(err <= PERSISTENT_BOUND[sp["precision"]]), (sp, err)
    mixed = lib.Batch(specs[:2] + [dict(specs[0], precision="p64")])
    assert not mixed.set_persistent(True)
    mixed.close()
