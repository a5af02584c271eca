"""Benchmark: grid-point updates/s of one AT-DNS time step on GB300.

Workload (the paper's decaying-turbulence configuration at 256^3, Sec. 4 /
Table 3 shapes): 256^3 periodic (2 pi)^3 box, 8x8x8 virtual PEs of 32^3
points (N_B = 33 %), 4th-order AT stencils with random delays uniform on
{0, 1, 2} (L = 2) from the seeded Philox stream, AB2 with a fixed dt, FP64,
statistics reduced every step.  Input: the seeded solenoidal field
E(k) ~ k^4 exp(-2 (k/4)^2), M_t = 0.3 (synthetic; the paper's forced
stationary fields are not available).  A step is one full pass of the hot path
(delay map, AT ghost assembly with the write of the current level's ring
slabs, derivative sweeps, assembly, AB2 update, reductions).  The working set (~8 GB) is far larger than L2, so no L2
flush is needed between steps.

Arms:
  default            the CUDA library (FP64 headline, FP32-bulk variant);
  --impl reference   the FP64 numpy oracle on the host cores, on a bounded
                     sample of the same workload (48^3 with 2x2x2 PEs of 24^3).

Prints one JSON line (rank 0).
"""
import argparse
import json
import os
import statistics as pystats
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "grid-point RK-step updates/s and HBM roofline fraction, FP64 vs FP32-bulk"
UNIT = "grid-point updates/s"
N, PES, L, SEED = 256, 8, 2, 2024
MU0 = None          # set from the resolution rule kappa_max eta = 1.5 at t = 0
# timed steps of the ensemble (the workload's 200 steps per run)
BATCH_STEPS = 200
CFL_AT = 0.2        # min(0.5, 0.8 / f(L)), f(2) = 0.90*4 - 0.35*2 + 1 = 3.9 (Sec. 3.2)
# FP64 operations per grid point of the main kernel, counted from the method
# (FMA = 2; division, square root and power = 1 each): 90 for the flux
# divergence (15 first derivatives x 6), 84 for the second derivatives (12 x 7),
# 36 for the mixed derivatives (6 x 6), ~100 for the assembly, 25 for the
# update and ~40 for the statistics.
FLOP_MAIN = 390.0
# the 6th-order scheme adds one stencil pair to every first derivative
# (15 flux + 6 mixed: +3 flops each) and second derivative (12: +3 each)
FLOP_MAIN6 = 489.0
NB_FRAC = 1.0 - (28.0 / 32.0) ** 3
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12   # SMs x DFMA/clk/SM x 2 x max SM clock
# DRAM bytes (read + write) of one launch of the dominant kernel at the
# 256^3 workload with 8x8x8 PEs of 32^3, from a one-pass ncu capture of that
# launch (dram__bytes_read.sum + dram__bytes_write.sum):
# k_main<double, 2> (multi-pass FP64): 7.79 GB + 3.84 GB; k_fused2<32, 8, plain>
# (P32C): 1.25 GB + 1.04 GB; 6th order (multi-pass): k_main<double, 3>
# 10.90 GB + 4.05 GB, k_main<float, 3> (P32C) 3.46 GB + 1.15 GB.
K_MAIN_FP64_TRAFFIC_256 = 7.79e9 + 3.84e9
K_FUSED2_P32C_TRAFFIC_256 = 1.25e9 + 1.04e9
K_MAIN_FP64_O6_TRAFFIC_256 = 10.90e9 + 4.05e9
K_MAIN_P32C_O6_TRAFFIC_256 = 3.46e9 + 1.15e9


def set_workload(n, pes):
    global N, PES, NB_FRAC
    N, PES = n, pes
    nl = n // pes
    NB_FRAC = 1.0 - ((nl - 4.0) / nl) ** 3


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {"hbm_gbs": 6800.0, "_fallback": True}


def nb_frac(order):
    """N_B / N_T per PE for half width M = order / 2 (Eqs. (NT)-(NB))."""
    nl = N // PES
    return 1.0 - ((nl - order) / float(nl)) ** 3


STATE_WORDS = {"p64": (8, 4), "p32": (4, 4), "p32c": (4, 6)}   # (bytes, words moved per variable)


def ghost_ratio(order):
    """AT ghost points per grid point: 2M ghost planes per PE face pair in
    each of the three directions (M = order / 2), 2M / n_l per direction."""
    return 0.0 if PES == 1 else 3.0 * order / (N // PES)


def xface_ratio(order):
    """Points of the x-face slabs (the first and last M points of a PE along
    x) per grid point."""
    return 0.0 if PES == 1 else order / float(N // PES)


def step_bytes(prec, order=4):
    """Algorithmic HBM bytes per grid point of one AB2 step (the workload's
    per-point figure): read U and R^{n-1}, write U^{n+1} and R^n (4 x 5 values;
    6 x 5 with the low words of the compensated form), plus the FP64 slab ring
    at the N_B fraction, one write and T_l reads of 5 values (T_l = 3 at 4th
    order, 4 at 6th)."""
    elem, words = STATE_WORDS[prec]
    return words * 5 * elem + nb_frac(order) * 5 * 8 * (1 + (3 if order == 4 else 4))


def algorithmic_bytes(prec, order=4, path="paired"):
    """HBM bytes per grid point that the step's main kernel must move.

    One-pass FP32 kernels (fused, paired): read U, R^{n-1} and write U^{n+1},
    R^n (P32C also reads and writes the low words of U); read the 9 ghost
    quantities (5 fluxes, u, v, w, T) of every AT ghost point; write the
    x-face slabs of U^{n+1} (with their low words in P32C) that the next
    step's ghost kernel reads.
    The FP64 multi-pass k_main: read the 16 primitive/flux arrays PQ, the 12
    gradients G, U and R^{n-1}, the ghost quantities; write U^{n+1} and R^n.
    The FP64 slab ring (one write and T_l reads of 5 variables at the N_B
    fraction) is the ghost kernel's traffic, not the main kernel's."""
    elem, words = STATE_WORDS[prec]
    ghosts = ghost_ratio(order) * 9 * elem
    if prec == "p64" or path == "multipass":
        return (16 + 12) * elem + words * 5 * elem + ghosts
    return words * 5 * elem + ghosts + xface_ratio(order) * 5 * elem * (2 if prec == "p32c" else 1)


class Clocks:
    """nvidia-smi sampler running during the timed region."""

    def __init__(self, out):
        self.out = out
        self.p = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.out, "w")
            self.p = subprocess.Popen(["nvidia-smi", "--query-gpu=" + q, "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()
            self.f.close()

    def summary(self, dev=0):
        rows = []
        try:
            for line in open(self.out):
                parts = [t.strip() for t in line.split(",")]
                if len(parts) < 9 or parts[0] != str(dev):
                    continue
                rows.append(parts)
        except Exception:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": pystats.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(ms, dist=None, device="cpu"):
    """Slowest rank's time (the job's time); identity on one process."""
    if dist is None:
        return float(ms)
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world, points, steps, ms):
    """Whole-job updates/s: every rank advances its own replica of `points`."""
    return world * points * steps / (ms / 1e3)


ORACLE_N, ORACLE_PES = 48, 2
ORACLE_BASELINE_STEPS = 10     # timed steps of the cpu_baseline sample (about 12 s on 16 host cores)


def _oracle_worker(steps, warmup, n, pes, seed, barrier, out):
    """One host core: the FP64 oracle, as it stands, stepping its own copy of
    the bounded sample (single-threaded numpy)."""
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"
    sys.path.insert(0, ROOT)
    from oracle import ns
    from paper_2003_10561_gb300 import synth
    U0 = synth.initial_state((n, n, n), k0=4.0, mach_t=0.3, seed=seed)
    cfg = ns.Config(n=(n, n, n), pes=(pes, pes, pes), mu0=0.01, max_delay=L, seed=SEED + seed)
    cfg.dt = ns.dt_from_cfl(cfg, U0, CFL_AT)
    hist = synth.history(U0, cfg.n_levels, eps=1e-3, seed=3 + seed)
    run = ns.Run.start(cfg, None, ns.RANDOM, step=cfg.n_levels + 2, history=hist)
    for _ in range(warmup):
        run.step()
    barrier.wait()
    t0 = time.perf_counter()
    for _ in range(steps):
        run.step()
    out.put(time.perf_counter() - t0)


def oracle_rate(steps, warmup, n=ORACLE_N, pes=ORACLE_PES, workers=None):
    """The FP64 oracle on all host cores: one spawned process per core, each
    stepping its own copy of an n^3 sample of the workload; the rate is the
    points all processes advanced over the slowest process's time.  Returns
    (rate, elapsed seconds, processes)."""
    import multiprocessing as mp
    workers = workers or os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    barrier = ctx.Barrier(workers)
    out = ctx.Queue()
    procs = [ctx.Process(target=_oracle_worker, args=(steps, warmup, n, pes, i, barrier, out), daemon=True)
             for i in range(workers)]
    for p_ in procs:
        p_.start()
    els = [out.get() for _ in procs]
    for p_ in procs:
        p_.join()
    el = max(els)
    return workers * n ** 3 * steps / el, el, workers


def run_reference(args, world, rank):
    if rank != 0:
        return 0
    steps = max(1, args.steps)
    warm = max(0, args.warmup)
    rate, el, cores = oracle_rate(steps, warm)
    sample = ("FP64 numpy oracle, one process per host core (%d), each taking AB2 steps of its own 48^3 box with "
              "2x2x2 PEs of 24^3 points, random delays L = 2 (the workload's method at a size the oracle "
              "finishes in seconds)" % cores)
    line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": args.gpus,
            "steps": steps, "warmup": warm, "ms_per_step": 1e3 * el / steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(world),
            "cpu_baseline": {"kind": "oracle", "value": rate, "unit": UNIT, "cores": cores, "sample": sample},
            "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def workload_config(world):
    nl = N // PES
    return {"workload": "decaying turbulence %d^3, %dx%dx%d virtual PEs (%d^3 each, N_B %.1f%%), 4th-order AT "
                        "stencils, random delays {0,1,2} (L=2), AB2, stats every step" % (N, PES, PES, PES, nl,
                                                                                        100 * NB_FRAC),
            "grid": [N, N, N], "pes": [PES, PES, PES], "max_delay": L, "delay_mode": "random",
            "boundary_fraction": NB_FRAC, "integrator": "AB2",
            "parallelism": "replicas" if world > 1 else "single",
            "l2": "working set %.1f GB >> 129 MB L2; no flush needed" % (N ** 3 * 5 * 8 * 12 / 1e9)}


def make_solver(at_dns, precision, stream, mu0, path="auto", order=4, **kw):
    # the cubic 6th-order weights shrink the stable CFL further: half the
    # 4th-order value (the step's cost does not depend on dt)
    cfl = CFL_AT if order == 4 else 0.5 * CFL_AT
    return at_dns.Solver(n=(N, N, N), pes=(PES, PES, PES), precision=precision, stream=stream, path=path,
                         gamma=1.4, prandtl=0.7, visc_exp=0.76, mu0=mu0, cfl=cfl, dt=0.0,
                         max_delay=L, seed=SEED, stats_every=1, order=order, **kw)


def timed_steps(s, stream, steps, warmup, torch, profile=False):
    """Device time of `steps` steps (CUDA events on the handle's stream; the
    library replays a captured one-step graph), then -- if asked -- the same
    number of steps launched kernel by kernel with an event pair around every
    launch, for the per-kernel times."""
    s.step(warmup, "random")
    s.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    s.step(steps, "random")
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    kt = {}
    if profile:
        s.profile(True)
        s.step(steps, "random")
        kt = s.kernel_times()
        s.profile(False)
    return ms, kt


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--grid", type=int, default=N, help="points per direction (profiling cases)")
    ap.add_argument("--pes", type=int, default=PES, help="virtual PEs per direction")
    ap.add_argument("--precision", default="both", choices=["both", "p64", "p32c", "p32"],
                    help="both: FP64 and the FP32-bulk form (P32C: FP32 stencils, compensated FP32 update, "
                         "FP64 ring and reductions)")
    ap.add_argument("--path", default="auto", choices=["auto", "multipass", "fused", "paired"])
    ap.add_argument("--order", default="both", choices=["both", "4", "6"],
                    help="spatial order of the AT scheme (4: headline; 6: Table B (1,6)/(2,6))")
    ap.add_argument("--no-tune", action="store_true",
                    help="keep the AUTO kernel path instead of the autotuner's pick")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-ensemble leg")
    ap.add_argument("--clocks-dir", default=None,
                    help="directory for the raw nvidia-smi clock samples (default: the system temp directory)")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the internal-energy / Sutherland leg")
    args = ap.parse_args()
    set_workload(args.grid, args.pes)
    args.warmup = max(args.warmup, 3)
    world, rank, local = dist_setup()

    if args.impl == "reference":
        return run_reference(args, world, rank)

    import numpy as np
    import torch
    torch.cuda.set_device(local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
        pg = dist
    from paper_2003_10561_gb300 import at_dns, synth
    at_dns.load()

    mu0 = synth.mu0_for_resolution((N, N, N), k0=4.0, mach_t=0.3, seed=0)
    U0 = synth.initial_state((N, N, N), k0=4.0, mach_t=0.3, seed=0)
    stream = torch.cuda.Stream()
    res = {}
    clocks = Clocks(os.path.join(args.clocks_dir or tempfile.gettempdir(), "bench_clocks_rank%d.csv" % rank))
    precs = ("p64", "p32c") if args.precision == "both" else (args.precision,)
    orders = (4, 6) if args.order == "both" else (int(args.order),)
    legs = [(p, o) for o in orders for p in precs]
    for prec, order in legs:
        key = prec if order == 4 else prec + "_o6"
        s = make_solver(at_dns, prec, stream.cuda_stream, mu0, args.path if order == 4 else "auto", order)
        s.set_state(U0)
        s.step(at_dns.at_dns_get_info(s.h).n_levels + 1, "random")   # past the synchronous start-up
        if not args.no_tune and args.path == "auto":
            s.tune("random", trials=3)    # kernel path, tile and z chunk from the autotuner
        if pg:
            pg.barrier()
        if key == legs[0][0] + ("" if legs[0][1] == 4 else "_o6"):
            with clocks:
                ms, kt = timed_steps(s, stream, args.steps, args.warmup, torch, profile=True)
        else:
            ms, kt = timed_steps(s, stream, args.steps, args.warmup, torch, profile=True)
        ms = max_over_ranks(ms, pg, "cuda")
        st = s.stats()
        res[key] = {"ms": ms, "kt": kt, "stats": st, "info": s.info(), "order": order, "prec": prec,
                    "dtype": "f64" if prec == "p64" else "f32"}
        # kernels in the timed region: every replayed step plus the health reset
        res[key]["launches"] = args.steps * res[key]["info"]["kernels_per_step"] + 1
        res[key]["path"] = {at_dns.AT_DNS_PATH_FUSED: "fused", at_dns.AT_DNS_PATH_PAIRED: "paired"}.get(
            res[key]["info"]["kernel_path"], "multipass")
        res[key]["tile"] = res[key]["info"]["tile"]
        # end to end through the public API with host buffers: per step, upload
        # U^n from pinned host memory (as the state of step n), step, read
        # U^{n+1} back into pinned host memory and the statistics record
        if key == "p64" and not args.no_e2e:
            host = torch.from_numpy(U0.copy()).pin_memory()
            back = torch.empty_like(host).pin_memory()
            nlev = at_dns.at_dns_get_info(s.h).n_levels
            e2e_steps = max(20, args.steps)
            s.set_history(host[None], nlev + 3)
            s.step(1, "random")
            s.get_state(back)
            s.stats()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for k in range(e2e_steps):
                s.set_history(host[None], nlev + 3 + k)
                s.step(1, "random")
                s.get_state(back)
                s.stats()
            el = max_over_ranks((time.perf_counter() - t0) * 1e3, pg, "cuda") / 1e3   # the slowest rank's
            res["e2e"] = {"value": world * N ** 3 * e2e_steps / el, "unit": UNIT,
                          "h2d_bytes_per_step": int(U0.nbytes),
                          "d2h_bytes_per_step": int(U0.nbytes) + int(ctypes_stats_size(at_dns)),
                          "steps": e2e_steps,
                          "per_step": "set_history(U^n from pinned host) + step(1) + get_state(U^{n+1} to pinned "
                                      "host) + stats()"}
        s.close()

    # synchronous low-storage RK3 (three right-hand sides per step), FP64
    if not args.no_variants and "p64" in res:
        s = make_solver(at_dns, "p64", stream.cuda_stream, mu0, "auto", 4, integrator=at_dns.AT_DNS_RK3)
        s.set_state(U0)
        s.step(2, "sync")
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        s.step(args.warmup, "sync")
        torch.cuda.synchronize()
        e0.record(stream)
        s.step(args.steps, "sync")
        e1.record(stream)
        torch.cuda.synchronize()
        res["rk3"] = {"ms": max_over_ranks(e0.elapsed_time(e1), pg, "cuda")}
        s.close()

    # the paper's own internal-energy form (Eq. (ie)) with Sutherland viscosity,
    # FP64, same workload: its step time beside the headline form's
    if not args.no_variants and "p64" in res:
        s = make_solver(at_dns, "p64", stream.cuda_stream, mu0, "auto", 4, energy_form=at_dns.AT_DNS_ENERGY_INTERNAL,
                        visc_law=at_dns.AT_DNS_VISC_SUTHERLAND)
        Ui = U0.copy()
        rho = U0[0]
        Ui[4] = U0[4] - 0.5 * (U0[1] ** 2 + U0[2] ** 2 + U0[3] ** 2) / rho   # rho e
        s.set_state(Ui)
        s.step(at_dns.at_dns_get_info(s.h).n_levels + 1, "random")
        ms, kt = timed_steps(s, stream, args.steps, args.warmup, torch, profile=False)
        ms = max_over_ranks(ms, pg, "cuda")
        res["variant"] = {"ms": ms}
        s.close()

    # batched ensemble: 64 independent decaying runs of uneven sizes advanced by
    # one graph launch per step (FP32-bulk, random delays, each member on the
    # path the batch autotuner picked), and by the opt-in persistent single
    # launch per step
    if not args.no_batch and N == 256:
        specs, states = [], []
        # mu0 by the resolution rule kappa_max eta = 1.5 of each member's spectrum:
        # <omega^2>^(1/2) grows linearly with M_t, so the rule is evaluated once
        # per (grid, k0) at M_t = 1 and scaled by the member's M_t
        mu_of = {(nb, k0): synth.mu0_for_resolution((nb,) * 3, k0=k0, mach_t=1.0, seed=0)
                 for nb in (32, 48, 64, 96, 128) for k0 in (3.0, 4.0, 6.0)}
        for i in range(64):
            nb = (32, 48, 64, 96, 128)[i % 5]
            k0 = (3.0, 4.0, 6.0)[i % 3]
            mt = 0.1 + 0.4 * i / 63.0
            specs.append(dict(n=(nb, nb, nb), pes=(nb // 16,) * 3, precision="p32c", gamma=1.4, prandtl=0.7,
                              visc_exp=0.76, mu0=mu_of[(nb, k0)] * mt, cfl=CFL_AT, dt=0.0, max_delay=L, seed=i,
                              stats_every=1))
            states.append(synth.initial_state((nb,) * 3, k0=k0, mach_t=mt, seed=i))
        bstream = torch.cuda.Stream()
        batch = at_dns.Batch(specs, stream=bstream.cuda_stream)
        for m, U in zip(batch.members, states):
            m.set_state(U)
        batch.step(6, "random")
        batch.tune("random", trials=2)     # tile shapes from the batch autotuner (states kept)
        timed = {}
        bsteps = BATCH_STEPS
        for persistent in (False, True):   # the graph of member branches, then the persistent launch
            batch.set_persistent(persistent)
            batch.step(args.warmup, "random")
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(bstream)
            batch.step(bsteps, "random")
            e1.record(bstream)
            torch.cuda.synchronize()
            timed[persistent] = (max_over_ranks(e0.elapsed_time(e1), pg, "cuda"), batch.persistent)
        bpts = float(sum(sp["n"][0] ** 3 for sp in specs))
        res["batch"] = {"ms": timed[True][0], "pts": bpts, "persistent": timed[True][1], "ms_graph": timed[False][0],
                        "steps": bsteps}
        batch.close()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, el, cores = oracle_rate(ORACLE_BASELINE_STEPS, 1)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": "%d AB2 steps (after 1 warm-up) of the FP64 numpy oracle in each of %d processes (one "
                         "per host core), each on its own 48^3 box with 2x2x2 PEs of 24^3 points, random delays "
                         "L = 2; %.1f s timed (slowest process)" % (ORACLE_BASELINE_STEPS, cores, el)}

    if rank != 0:
        return 0
    pk = peaks()
    pts = float(N ** 3)
    p64 = res.get("p64")
    p32 = res.get("p32c") or res.get("p32")
    head = p64 or p32 or res.get("p64_o6") or res.get("p32c_o6") or res.get("p32_o6")
    value = job_rate(world, pts, args.steps, head["ms"])
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": head["ms"] / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if head in (p64, res.get("p64_o6")) else "f32",
        "data": "synthetic", "config": workload_config(world),
        "kernel_ms_per_step": {k: v[1] / v[0] for k, v in head["kt"].items()},
        "e2e": res.get("e2e"),
        "cpu_baseline": cpu,
        "clocks": clocks.summary(local),
        "gpu_launches": head["launches"],
        "rhs_per_s": value,
        "kernel_path": head["path"],
        "tile": head["tile"],
        "order": head["order"],
    }
    rep = {k: leg_report(r, world, pts, args.steps, pk) for k, r in res.items()
           if k not in ("e2e", "variant", "rk3", "batch")}
    if "batch" in res:
        bt = res["batch"]
        line["batch_ensemble"] = {
            "value": job_rate(world, bt["pts"], bt["steps"], bt["ms_graph"]), "unit": UNIT, "dtype": "f32",
            "ms_per_step": bt["ms_graph"] / bt["steps"], "members": 64, "steps": bt["steps"],
            "form": "one graph launch per step, each member on its own branch and on the path the batch "
                    "autotuner picked",
            "persistent_form": {"value": job_rate(world, bt["pts"], bt["steps"], bt["ms"]),
                                "ms_per_step": bt["ms"] / bt["steps"],
                                "one_persistent_launch_per_step": bt["persistent"],
                                "note": "opt-in: one cooperative kernel launch per step over the members' ghost "
                                        "items and paired-kernel tiles"},
            "workload": "64 decaying runs, grids {32,48,64,96,128}^3 by member, PEs of 16^3, M_t 0.1..0.5, "
                        "k0 in {3,4,6}, seeds 0..63, FP32-bulk (P32C), random delays L = 2"}
    if "rk3" in res:
        line["rk3_sync"] = {
            "value": job_rate(world, pts, args.steps, res["rk3"]["ms"]), "unit": UNIT, "dtype": "f64",
            "ms_per_step": res["rk3"]["ms"] / args.steps,
            "workload": "the headline box and state, synchronous (no delays), three-stage low-storage RK3"}
    if "variant" in res:
        line["variant_rhoe_sutherland"] = {
            "value": job_rate(world, pts, args.steps, res["variant"]["ms"]), "unit": UNIT, "dtype": "f64",
            "ms_per_step": res["variant"]["ms"] / args.steps,
            "workload": "the headline workload with the internal-energy form (Eq. (ie)) and Sutherland viscosity"}
    line["roofline"] = rep[[k for k in res if res[k] is head][0]]["roofline"]
    if p32 and p32 is not head:
        blk = rep[p32["prec"]]
        blk["form"] = {"p32c": "P32C: FP32 state and stencils, compensated (TwoSum hi + lo) FP32 update, FP64 slab "
                               "ring, compensated FP32 sums within a block and FP64 across blocks",
                       "p32": "P32: FP32 state, stencils and update; FP64 slab ring and reductions"}[p32["prec"]]
        if p64:
            blk["rel_err_vs_fp64"] = {k: abs(p32["stats"][k] - p64["stats"][k]) / abs(p64["stats"][k])
                                      for k in ("tke", "dissipation")}
        line["fp32_bulk"] = blk
    o6 = {k[:-3]: rep[k] for k in ("p64_o6", "p32c_o6", "p32_o6") if k in rep and res[k] is not head}
    if o6:
        line["order6"] = dict(o6, workload="the same box, PEs, delays and state with the 6th-order AT scheme "
                                            "(Table B (1,6)/(2,6), T_l = 4, N_B %.1f%%)" % (100 * nb_frac(6)))
    print(json.dumps(line), flush=True)
    return 0


def leg_report(r, world, pts, steps, pk):
    """Throughput, per-kernel times and the roofline of the main kernel of one
    measured (precision, order) leg.

    The HBM roofline takes the step's algorithmic bytes per point (step_bytes)
    times the points of one launch over the main kernel's average launch time.
    Beside it: the bytes the main kernel itself must move (algorithmic_bytes;
    in this design the ghost kernel moves the FP64 slab ring) with that
    kernel's own fraction, and the whole step's fraction (step bytes over the
    step time)."""
    order = r["order"]
    main = r["kt"].get("main", (1, 1.0))
    t_main = main[1] / main[0] / 1e3
    t_step = r["ms"] / steps / 1e3
    hbm = pk.get("hbm_gbs", 6800.0)
    sb = step_bytes(r["prec"], order)
    kb = algorithmic_bytes(r["prec"], order, r["path"])
    hbm_fields = {"peak": pk.get("hbm_gbs"), "unit": "GB/s", "bytes_per_point": sb,
                  "kernel_bytes_per_point": kb, "kernel_frac": kb * pts / t_main / 1e9 / hbm,
                  "step_frac": sb * pts / t_step / 1e9 / hbm}
    if r["dtype"] == "f64":
        flops = FLOP_MAIN if order == 4 else FLOP_MAIN6
        achieved = flops * pts / t_main / 1e12
        traffic = None
        if N == 256 and PES == 8 and r["path"] == "multipass":
            traffic = K_MAIN_FP64_TRAFFIC_256 if order == 4 else K_MAIN_FP64_O6_TRAFFIC_256
        roof = {"bound": "alu", "kernel": "k_main (FP64, order %d)" % order, "achieved": achieved,
                "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS,
                "traffic": traffic, "flop_per_point": flops,
                "note": "FP64 peak derived: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz "
                        "(an FMA probe measured 1.20 TFLOP/s)"}
        # the same kernel against the HBM roof
        gbs = sb * pts / t_main / 1e9
        roof["hbm"] = dict(hbm_fields, achieved=gbs, frac=gbs / hbm)
    else:
        achieved = sb * pts / t_main / 1e9
        kname = {"fused": "k_fused", "paired": "k_fused2"}.get(r["path"], "k_main")
        traffic = None
        if N == 256 and PES == 8 and r["prec"] == "p32c":
            if order == 4 and r["path"] == "paired" and list(r["tile"]) == [32, 8, 32]:
                traffic = K_FUSED2_P32C_TRAFFIC_256
            elif order == 6 and r["path"] == "multipass":
                traffic = K_MAIN_P32C_O6_TRAFFIC_256
        roof = dict(hbm_fields, bound="hbm", kernel="%s (FP32, order %d)" % (kname, order), achieved=achieved,
                    frac=achieved / hbm, traffic=traffic)
    return {"value": job_rate(world, pts, steps, r["ms"]), "unit": UNIT, "kernel_path": r["path"], "tile": r["tile"],
            "ms_per_step": r["ms"] / steps, "dtype": r["dtype"], "roofline": roof,
            "kernel_ms_per_step": {k: v[1] / v[0] for k, v in r["kt"].items()}}


def ctypes_stats_size(at_dns):
    import ctypes
    return ctypes.sizeof(at_dns.at_dns_stats_t)


if __name__ == "__main__":
    sys.exit(main())
