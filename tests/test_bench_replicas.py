"""The multi-GPU path of bench.py is replicas only: every rank advances its own
copy of the workload, ranks meet at a barrier, the job time is the slowest
rank's and the job rate counts all ranks' points.  Checked here with two gloo
ranks on the CPU (no GPU, no collective on the data path)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    dist.barrier()
    ms = 10.0 * (rank + 1)                 # the ranks' own timed regions differ
    job_ms = bench.max_over_ranks(ms, dist, "cpu")
    out[rank] = (job_ms, bench.job_rate(world, 64 ** 3, 5, job_ms))
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_take_slowest_rank_and_sum_points():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
    assert out[0][0] == out[1][0] == 20.0
    assert out[0][1] == pytest.approx(2 * 64 ** 3 * 5 / 0.020)


def test_single_process_identity():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.job_rate(1, 100, 4, 2.0) == pytest.approx(200000.0)


def test_algorithmic_bytes_and_roofline_fields():
    """Algorithmic bytes per point at 8^3 PEs of 32^3 (N_B = 1 - (28/32)^3).
    The step's figure (the roofline's): 4 x 5 values of U and R (6 x 5 in the
    compensated FP32 form, which also moves the low words of U) plus the FP64
    slab ring, one write and T_l = 3 reads of 5 values at the N_B fraction.
    The main kernel's own figure: one-pass FP32 kernel -- U, R (and low
    words), the 9 ghost quantities of the 3 x 2M / 32 = 0.375 AT ghost points
    per point, the x-face slabs of U^{n+1} (2M / 32 = 0.125 points per point,
    with their low words in P32C); FP64 multi-pass k_main -- the 16 PQ and 12 G
    arrays, 4 x 5 values of U and R, the ghost quantities.  The FP64 leg
    reports its FP64-pipe fraction and, beside it, its HBM fraction."""
    import bench
    bench.set_workload(256, 8)
    nb = 1.0 - (28.0 / 32.0) ** 3
    ring = nb * 5 * 8 * 4
    assert bench.step_bytes("p64") == pytest.approx(160.0 + ring)
    assert bench.step_bytes("p32") == pytest.approx(80.0 + ring)
    assert bench.step_bytes("p32c") == pytest.approx(120.0 + ring)
    assert round(bench.step_bytes("p64"), 1) == 212.8 and round(bench.step_bytes("p32c"), 1) == 172.8
    assert bench.ghost_ratio(4) == pytest.approx(0.375) and bench.xface_ratio(4) == pytest.approx(0.125)
    assert bench.algorithmic_bytes("p32c") == pytest.approx(120.0 + 0.375 * 36 + 0.125 * 40)
    assert bench.algorithmic_bytes("p32") == pytest.approx(80.0 + 0.375 * 36 + 0.125 * 20)
    assert bench.algorithmic_bytes("p64", 4, "multipass") == pytest.approx(28 * 8 + 160.0 + 0.375 * 72)
    assert round(bench.algorithmic_bytes("p32c"), 1) == 138.5
    assert round(bench.algorithmic_bytes("p64", 4, "multipass"), 1) == 411.0
    pts, steps = 256 ** 3, 5
    r64 = {"order": 4, "kt": {"main": (steps, 5 * 11.0)}, "dtype": "f64", "prec": "p64", "path": "multipass",
           "tile": [0, 0, 0], "ms": steps * 14.0}
    roof = bench.leg_report(r64, 1, pts, steps, {"hbm_gbs": 6801.7})["roofline"]
    assert roof["bound"] == "alu" and roof["unit"] == "TFLOP/s"
    assert roof["achieved"] == pytest.approx(bench.FLOP_MAIN * pts / 11e-3 / 1e12)
    assert roof["frac"] == pytest.approx(roof["achieved"] / bench.FP64_PEAK_TFLOPS)
    assert roof["hbm"]["frac"] == pytest.approx(bench.step_bytes("p64") * pts / 11e-3 / 1e9 / 6801.7)
    assert roof["hbm"]["kernel_frac"] == pytest.approx(411.0 * pts / 11e-3 / 1e9 / 6801.7)
    r32 = dict(r64, dtype="f32", prec="p32c", path="paired", tile=[32, 8, 32], kt={"main": (steps, 5 * 1.5)},
               ms=steps * 1.7)
    roof = bench.leg_report(r32, 1, pts, steps, {"hbm_gbs": 6801.7})["roofline"]
    assert roof["bound"] == "hbm" and roof["unit"] == "GB/s" and roof["bytes_per_point"] == bench.step_bytes("p32c")
    assert roof["frac"] == pytest.approx(bench.step_bytes("p32c") * pts / 1.5e-3 / 1e9 / 6801.7)
    assert roof["kernel_frac"] == pytest.approx(138.5 * pts / 1.5e-3 / 1e9 / 6801.7)
    assert roof["step_frac"] == pytest.approx(bench.step_bytes("p32c") * pts / 1.7e-3 / 1e9 / 6801.7)
    assert roof["traffic"] == bench.K_FUSED2_P32C_TRAFFIC_256


def test_oracle_baseline_uses_every_core():
    """The CPU baseline runs one oracle process per core (spawned) and counts
    the points of all of them over the slowest one's time."""
    import bench
    rate, el, cores = bench.oracle_rate(1, 0, n=12, pes=2, workers=2)
    assert cores == 2 and el > 0
    assert rate == pytest.approx(2 * 12 ** 3 / el)
