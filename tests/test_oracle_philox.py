"""Pins of the oracle's Philox4x32-10 against the published known-answer
vectors (tests/golden/philox4x32_10_kat.txt) and against Triton's independent
Philox implementation run by its CPU interpreter."""
import os

import numpy as np
import pytest

from oracle.philox import philox4x32_10, split_seed

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        rows.append([int(t, 16) for t in line.split()])
    return rows


def test_known_answer_vectors():
    rows = _kat()
    assert len(rows) == 3
    for r in rows:
        out = philox4x32_10(*r[:6])
        assert [int(v) for v in out] == r[6:]


def test_vectorised_matches_scalar():
    c0 = np.arange(7, dtype=np.uint64)
    out = philox4x32_10(c0, 5, 6, 0x4154, 0x1234, 0x5678)
    for i in range(7):
        one = philox4x32_10(i, 5, 6, 0x4154, 0x1234, 0x5678)
        assert all(int(out[w][i]) == int(one[w]) for w in range(4))


def test_split_seed():
    assert split_seed(0x0123456789ABCDEF) == (0x89ABCDEF, 0x01234567)


def test_against_triton_interpreter():
    """Triton's own Philox (tl.philox, 10 rounds, key = (seed lo, seed hi))
    executed by its numpy interpreter on the CPU."""
    os.environ.setdefault("TRITON_INTERPRET", "1")
    if os.environ.get("TRITON_INTERPRET") != "1":
        pytest.skip("Triton interpreter not selected")
    torch = pytest.importorskip("torch")
    triton = pytest.importorskip("triton")
    import triton.language as tl

    @triton.jit
    def k(out_ptr, seed, c1, c2, c3):
        offs = tl.arange(0, 8)
        c0 = offs.to(tl.uint32)
        a, b, c, d = tl.philox(seed, c0, c1 + 0 * c0, c2 + 0 * c0, c3 + 0 * c0)
        tl.store(out_ptr + offs * 4 + 0, a.to(tl.int64))
        tl.store(out_ptr + offs * 4 + 1, b.to(tl.int64))
        tl.store(out_ptr + offs * 4 + 2, c.to(tl.int64))
        tl.store(out_ptr + offs * 4 + 3, d.to(tl.int64))

    seed = 0x1F2E3D4C5B6A7988
    out = torch.zeros(32, dtype=torch.int64)
    try:
        k[(1,)](out, seed, 11, 22, 0x4154)
    except Exception as e:  # interpreter unavailable in this environment
        pytest.skip("triton interpreter failed: %s" % e)
    got = (out.numpy() & 0xFFFFFFFF).reshape(8, 4)
    k0, k1 = split_seed(seed)
    ref = philox4x32_10(np.arange(8, dtype=np.uint64), 11, 22, 0x4154, k0, k1)
    for w in range(4):
        assert np.array_equal(got[:, w], ref[w].astype(np.int64))
