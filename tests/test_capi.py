"""CPU checks of the C ABI: the library builds and loads without a GPU, exports
every function include/at_dns.h declares, its structs have the header's
layout, and configuration errors are caught before any device work."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

from paper_2003_10561_gb300 import at_dns, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "at_dns.h")


@pytest.fixture(scope="module")
def lib():
    return at_dns.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(at_dns_\w+)\s*\(", text)))


def test_every_declared_symbol_exported(lib):
    names = declared_functions()
    assert len(names) >= 12
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(at_dns._SIGS)


def _c_layout():
    src = r'''
#include <stdio.h>
#include <stddef.h>
#include "at_dns.h"
#define F(T, m) printf(#T " " #m " %zu\n", offsetof(T, m));
int main(void) {
  printf("at_dns_config_t size %zu\n", sizeof(at_dns_config_t));
  printf("at_dns_stats_t size %zu\n", sizeof(at_dns_stats_t));
  printf("at_dns_info_t size %zu\n", sizeof(at_dns_info_t));
  F(at_dns_config_t, seed) F(at_dns_config_t, forcing) F(at_dns_config_t, f_seed)
  F(at_dns_config_t, precision) F(at_dns_config_t, stream) F(at_dns_config_t, kernel_path)
  F(at_dns_config_t, order) F(at_dns_info_t, order)
  F(at_dns_config_t, energy_form) F(at_dns_config_t, visc_law) F(at_dns_config_t, sutherland_s)
  F(at_dns_config_t, integrator) F(at_dns_config_t, pool) F(at_dns_config_t, pool_bytes)
  F(at_dns_config_t, extrapolate_state)
  F(at_dns_stats_t, mom) F(at_dns_stats_t, min_p) F(at_dns_stats_t, unstable)
  F(at_dns_info_t, n_levels) F(at_dns_info_t, device_bytes) F(at_dns_info_t, kernels_per_step)
  F(at_dns_info_t, kernel_path) F(at_dns_info_t, tile)
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "l.c")
        open(c, "w").write(src)
        exe = os.path.join(d, "l")
        subprocess.run(["gcc", "-I", os.path.dirname(HEADER), c, "-o", exe], check=True)
        return subprocess.run([exe], capture_output=True, text=True, check=True).stdout


def test_struct_layout_matches_header():
    out = _c_layout()
    types = {"at_dns_config_t": at_dns.at_dns_config_t, "at_dns_stats_t": at_dns.at_dns_stats_t,
             "at_dns_info_t": at_dns.at_dns_info_t}
    for line in out.strip().splitlines():
        T, m, v = line.split()
        if m == "size":
            assert ctypes.sizeof(types[T]) == int(v), line
        else:
            assert getattr(types[T], m).offset == int(v), line


def test_config_default(lib):
    cfg = at_dns.at_dns_config_default()
    assert list(cfg.n) == [32, 32, 32] and list(cfg.pes) == [1, 1, 1]
    assert cfg.gamma == 1.4 and cfg.prandtl == 0.7 and cfg.visc_exp == 0.76
    assert cfg.max_delay == 2 and cfg.comm_period == 3 and cfg.precision == at_dns.AT_DNS_P64
    assert cfg.order == 4 and cfg.energy_form == at_dns.AT_DNS_ENERGY_TOTAL
    assert cfg.visc_law == at_dns.AT_DNS_VISC_POWER and cfg.sutherland_s == 0.368


@pytest.mark.parametrize("field,value", [
    ("n", (4, 32, 32)), ("pes", (3, 1, 1)), ("pes", (8, 1, 1)), ("gamma", 1.0),
    ("max_delay", -1), ("comm_period", 0), ("precision", 7), ("prandtl", 0.0), ("kernel_path", 9),
    ("order", 5), ("order", 8), ("energy_form", 2), ("visc_law", 3), ("sutherland_s", 0.0), ("integrator", 2),
    ("extrapolate_state", 2),
])
def test_create_rejects_bad_config_without_gpu(lib, field, value):
    cfg = at_dns.at_dns_config_default()
    if field == "sutherland_s":
        cfg.visc_law = at_dns.AT_DNS_VISC_SUTHERLAND
    if isinstance(value, tuple):
        for i, v in enumerate(value):
            getattr(cfg, field)[i] = v
    else:
        setattr(cfg, field, value)
    h = ctypes.c_void_p()
    rc = lib.at_dns_create(ctypes.byref(cfg), ctypes.byref(h))
    assert rc == at_dns.AT_DNS_E_INVALID_ARG
    assert h.value is None
    assert at_dns.at_dns_last_error(None) != ""


@pytest.mark.parametrize("n,pes", [((6, 32, 32), (1, 1, 1)), ((36, 32, 32), (6, 1, 1))])
def test_create_rejects_sixth_order_below_seven_points_without_gpu(lib, n, pes):
    cfg = at_dns.make_config(n=n, pes=pes, order=6)
    h = ctypes.c_void_p()
    assert lib.at_dns_create(ctypes.byref(cfg), ctypes.byref(h)) == at_dns.AT_DNS_E_INVALID_ARG
    assert "order + 1" in at_dns.at_dns_last_error(None)


def test_null_arguments(lib):
    assert lib.at_dns_config_default(None) == at_dns.AT_DNS_E_INVALID_ARG
    assert lib.at_dns_create(None, None) == at_dns.AT_DNS_E_INVALID_ARG
    assert lib.at_dns_step(None, 1, 0) == at_dns.AT_DNS_E_INVALID_ARG
    assert lib.at_dns_rhs(None, 0, None, 0) == at_dns.AT_DNS_E_INVALID_ARG
    lib.at_dns_destroy(None)


def test_null_arguments_of_checkpoint_batch_and_selftest_calls(lib):
    """The checkpoint, batch and self-test entry points refuse null handles and
    buffers and out-of-range arguments before any device work."""
    import ctypes
    n = ctypes.c_int64(0)
    assert lib.at_dns_checkpoint_size(None, ctypes.byref(n)) == at_dns.AT_DNS_E_INVALID_ARG
    assert lib.at_dns_checkpoint_save(None, None, 0) == at_dns.AT_DNS_E_INVALID_ARG
    assert lib.at_dns_checkpoint_load(None, None, 0) == at_dns.AT_DNS_E_INVALID_ARG
    assert lib.at_dns_batch_step(None, 1, 0) == at_dns.AT_DNS_E_INVALID_ARG
    assert lib.at_dns_batch_persistent(None, 1, None) == at_dns.AT_DNS_E_INVALID_ARG
    g = ctypes.c_int32(0)
    assert lib.at_dns_wait_selftest(27, ctypes.byref(g)) == at_dns.AT_DNS_E_INVALID_ARG
    assert lib.at_dns_wait_selftest(-1, ctypes.byref(g)) == at_dns.AT_DNS_E_INVALID_ARG
    assert lib.at_dns_wait_selftest(10, None) == at_dns.AT_DNS_E_INVALID_ARG


def test_checkpoint_buffers_are_checked_by_the_binding():
    """Checkpoint buffers are C-contiguous uint8 arrays or tensors of at least
    the checkpoint's size; anything else is refused before the C call."""
    import numpy as np
    with pytest.raises(TypeError):
        at_dns._byte_ptr(np.zeros(16, dtype=np.float64), 8)
    with pytest.raises(TypeError):
        at_dns._byte_ptr(np.zeros(8, dtype=np.uint8), 16)
    with pytest.raises(TypeError):
        at_dns._byte_ptr(np.zeros((4, 8), dtype=np.uint8)[:, ::2], 8)
    with pytest.raises(TypeError):
        at_dns._byte_ptr([0] * 16, 8)
    a = np.zeros(32, dtype=np.uint8)
    assert at_dns._byte_ptr(a, 32) == (a.ctypes.data, at_dns.AT_DNS_HOST)
    torch = pytest.importorskip("torch")
    t = torch.zeros(32, dtype=torch.uint8)
    assert at_dns._byte_ptr(t, 32) == (t.data_ptr(), at_dns.AT_DNS_HOST)
    with pytest.raises(TypeError):
        at_dns._byte_ptr(torch.zeros(32, dtype=torch.float32), 8)


def test_checked_build_variant_is_separate():
    """The bounds-checked library is built apart (its own objects and file) with
    -DAT_DNS_CHECKS, and at_dns.load() picks it only when asked."""
    assert build.LIB_CHECKED != build.LIB and build.BUILD_CHECKED != build.BUILD
    assert os.path.dirname(build.LIB_CHECKED) == os.path.dirname(build.LIB)
    import inspect
    src = inspect.getsource(build.build)
    assert "-DAT_DNS_CHECKS" in src
    assert "AT_DNS_LIBRARY" in inspect.getsource(at_dns.load)


def test_build_is_in_tree():
    assert os.path.dirname(build.LIB) == os.path.join(ROOT, "paper_2003_10561_gb300")
    assert build.up_to_date()
