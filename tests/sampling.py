"""Sampled points and inputs of the full-size (256^3) parity case, shared by
the GPU test and the script that writes its extended-precision reference."""
import numpy as np

# the benchmark workload: 256^3, 8x8x8 PEs of 32^3, random delays with L = 2,
# evaluated at step 17 (past the synchronous start-up)
FULL_N, FULL_PES, FULL_L, FULL_STEP, FULL_SEED = (256, 256, 256), (8, 8, 8), 2, 17, 2024
FULL_KW = dict(mu0=0.004, dt=1e-3, max_delay=FULL_L, seed=FULL_SEED)


def sample_points(n, nloc, rng, count):
    """Random points plus PE face, edge and corner points and the ragged ends."""
    pts = set()
    for _ in range(count):
        pts.add(tuple(int(rng.integers(0, n[d])) for d in range(3)))
    special = [0, 1, nloc - 2, nloc - 1, nloc, nloc + 1, 2, nloc // 2]
    for a in special:
        for b in (0, 1, nloc - 1, 5):
            pts.add((a % n[0], b % n[1], (a + b) % n[2]))
            pts.add((b % n[0], a % n[1], 3 % n[2]))
    pts.add((n[0] - 1, n[1] - 1, n[2] - 1))
    return sorted(pts)


def full_size_points():
    return sample_points(FULL_N, FULL_N[0] // FULL_PES[0], np.random.default_rng(4), 120)


def full_size_history():
    """The seeded levels of the full-size case (the state and its past)."""
    from oracle import ns
    from paper_2003_10561_gb300 import synth
    U0 = synth.initial_state(FULL_N, k0=4.0, mach_t=0.3, seed=1)
    c = ns.Config(n=FULL_N, pes=FULL_PES, gamma=1.4, prandtl=0.7, visc_exp=0.76, **FULL_KW)
    return c, synth.history(U0, c.n_levels, eps=1e-2, seed=3)
