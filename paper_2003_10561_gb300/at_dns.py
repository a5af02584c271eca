"""Thin ctypes binding of the C ABI in include/at_dns.h (same names).

Argument marshalling only: every step of the solver runs in the CUDA library.
Arrays are passed as host pointers (C-contiguous numpy float64) or device
pointers (CUDA torch tensors, float64); the binding raises if the compiled
library is missing -- there is no other implementation behind it.
"""
import ctypes
import os

import numpy as np

from . import build as _build

AT_DNS_OK = 0
AT_DNS_E_INVALID_ARG = -1
AT_DNS_E_OOM = -2
AT_DNS_E_CUDA = -3
AT_DNS_E_UNSTABLE = -4
AT_DNS_E_UNSUPPORTED = -5
AT_DNS_E_STATE = -6
AT_DNS_E_TOO_LARGE = -7
AT_DNS_E_TIMEOUT = -8
AT_DNS_E_BOUNDS = -9
AT_DNS_NOALLOC_MAX_POINTS = 262144

AT_DNS_SYNC, AT_DNS_PERIODIC, AT_DNS_RANDOM, AT_DNS_FIXED, AT_DNS_ORDERED = 0, 1, 2, 3, 4
AT_DNS_P64, AT_DNS_P32, AT_DNS_P32C = 0, 1, 2
AT_DNS_HOST, AT_DNS_DEVICE = 0, 1
AT_DNS_PATH_AUTO, AT_DNS_PATH_MULTIPASS, AT_DNS_PATH_FUSED, AT_DNS_PATH_PAIRED = 0, 1, 2, 3
AT_DNS_ENERGY_TOTAL, AT_DNS_ENERGY_INTERNAL = 0, 1
AT_DNS_VISC_POWER, AT_DNS_VISC_SUTHERLAND = 0, 1
AT_DNS_AB2, AT_DNS_RK3 = 0, 1
PATHS = {"auto": AT_DNS_PATH_AUTO, "multipass": AT_DNS_PATH_MULTIPASS, "fused": AT_DNS_PATH_FUSED,
         "paired": AT_DNS_PATH_PAIRED}

MODES = {"sync": AT_DNS_SYNC, "periodic": AT_DNS_PERIODIC, "random": AT_DNS_RANDOM, "fixed": AT_DNS_FIXED,
         "ordered": AT_DNS_ORDERED}
PRECISIONS = {"p64": AT_DNS_P64, "p32": AT_DNS_P32, "p32c": AT_DNS_P32C}


class at_dns_config_t(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int32 * 3), ("pes", ctypes.c_int32 * 3),
        ("gamma", ctypes.c_double), ("prandtl", ctypes.c_double), ("mu0", ctypes.c_double),
        ("visc_exp", ctypes.c_double), ("dt", ctypes.c_double), ("cfl", ctypes.c_double),
        ("max_delay", ctypes.c_int32), ("comm_period", ctypes.c_int32), ("seed", ctypes.c_uint64),
        ("forcing", ctypes.c_int32), ("kf", ctypes.c_double), ("f_amp", ctypes.c_double),
        ("f_tcorr", ctypes.c_double), ("f_seed", ctypes.c_uint64),
        ("precision", ctypes.c_int32), ("stats_every", ctypes.c_int32), ("stream", ctypes.c_void_p),
        ("kernel_path", ctypes.c_int32), ("order", ctypes.c_int32),
        ("energy_form", ctypes.c_int32), ("visc_law", ctypes.c_int32), ("sutherland_s", ctypes.c_double),
        ("integrator", ctypes.c_int32), ("pool", ctypes.c_void_p), ("pool_bytes", ctypes.c_size_t),
        ("extrapolate_state", ctypes.c_int32),
    ]


class at_dns_stats_t(ctypes.Structure):
    _fields_ = [
        ("step", ctypes.c_int64), ("time", ctypes.c_double), ("dt", ctypes.c_double),
        ("mass", ctypes.c_double), ("mom", ctypes.c_double * 3), ("energy", ctypes.c_double),
        ("tke", ctypes.c_double), ("dissipation", ctypes.c_double),
        ("grad_m2", ctypes.c_double), ("grad_m3", ctypes.c_double), ("grad_m4", ctypes.c_double),
        ("skewness", ctypes.c_double), ("flatness", ctypes.c_double), ("enstrophy", ctypes.c_double),
        ("pressure_dilatation", ctypes.c_double), ("forcing_power", ctypes.c_double),
        ("urms", ctypes.c_double), ("mach_t", ctypes.c_double), ("max_wave_speed", ctypes.c_double),
        ("min_rho", ctypes.c_double), ("min_p", ctypes.c_double), ("unstable", ctypes.c_int32),
    ]

    def as_dict(self):
        out = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            out[name] = list(v) if name == "mom" else v
        return out


class at_dns_info_t(ctypes.Structure):
    _fields_ = [
        ("step", ctypes.c_int64), ("time", ctypes.c_double), ("dt", ctypes.c_double),
        ("n_levels", ctypes.c_int32), ("boundary_fraction", ctypes.c_double),
        ("device_bytes", ctypes.c_size_t), ("kernels_per_step", ctypes.c_int32),
        ("kernel_path", ctypes.c_int32), ("tile", ctypes.c_int32 * 3), ("order", ctypes.c_int32),
    ]


class at_dns_kernel_time_t(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 24), ("launches", ctypes.c_int64), ("total_ms", ctypes.c_double)]


_P = ctypes.c_void_p
_SIGS = {
    "at_dns_config_default": (ctypes.c_int, [ctypes.POINTER(at_dns_config_t)]),
    "at_dns_create": (ctypes.c_int, [ctypes.POINTER(at_dns_config_t), ctypes.POINTER(_P)]),
    "at_dns_set_state": (ctypes.c_int, [_P, _P, ctypes.c_int]),
    "at_dns_set_history": (ctypes.c_int, [_P, _P, ctypes.c_int32, ctypes.c_int64, ctypes.c_int]),
    "at_dns_get_state": (ctypes.c_int, [_P, _P, ctypes.c_int]),
    "at_dns_rhs": (ctypes.c_int, [_P, ctypes.c_int32, _P, ctypes.c_int]),
    "at_dns_step": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32]),
    "at_dns_stats": (ctypes.c_int, [_P, ctypes.POINTER(at_dns_stats_t)]),
    "at_dns_get_delay_map": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_int32, _P]),
    "at_dns_get_info": (ctypes.c_int, [_P, ctypes.POINTER(at_dns_info_t)]),
    "at_dns_profile": (ctypes.c_int, [_P, ctypes.c_int32]),
    "at_dns_kernel_times": (ctypes.c_int, [_P, ctypes.POINTER(at_dns_kernel_time_t), ctypes.c_int32,
                                           ctypes.POINTER(ctypes.c_int32)]),
    "at_dns_synchronize": (ctypes.c_int, [_P]),
    "at_dns_set_kernel_path": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]),
    "at_dns_tune": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(ctypes.c_double)]),
    "at_dns_batch_create": (ctypes.c_int, [ctypes.POINTER(at_dns_config_t), ctypes.c_int32, _P, ctypes.POINTER(_P)]),
    "at_dns_batch_member": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(_P)]),
    "at_dns_batch_step": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32]),
    "at_dns_batch_tune": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32]),
    "at_dns_batch_persistent": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]),
    "at_dns_wait_selftest": (ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]),
    "at_dns_checkpoint_size": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int64)]),
    "at_dns_checkpoint_save": (ctypes.c_int, [_P, ctypes.c_void_p, ctypes.c_int]),
    "at_dns_checkpoint_load": (ctypes.c_int, [_P, ctypes.c_void_p, ctypes.c_int]),
    "at_dns_batch_last_error": (ctypes.c_char_p, [_P]),
    "at_dns_batch_destroy": (None, [_P]),
    "at_dns_rhs_noalloc": (ctypes.c_int, [ctypes.POINTER(ctypes.c_int32), ctypes.c_double, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_double, _P, _P, _P]),
    "at_dns_last_error": (ctypes.c_char_p, [_P]),
    "at_dns_destroy": (None, [_P]),
}

_lib = None


def library_path():
    return _build.LIB


def load(build_if_missing=True):
    """Load libat_dns.so (building it in-tree first if asked and needed).  With
    AT_DNS_LIBRARY=checked in the environment: the bounds-checked build
    libat_dns_checked.so instead (index checks in the kernels)."""
    global _lib
    if _lib is not None:
        return _lib
    checked = os.environ.get("AT_DNS_LIBRARY") == "checked"
    path = _build.LIB_CHECKED if checked else _build.LIB
    if build_if_missing and not _build.up_to_date(checked):
        _build.build(checked=checked)
    if not os.path.exists(path):
        raise ImportError("%s is not built (run paper_2003_10561_gb300.build.build())" % os.path.basename(path))
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class AtDnsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("at_dns error %d: %s" % (code, msg))
        self.code = code


def _check(rc, h=None):
    if rc != AT_DNS_OK:
        msg = load().at_dns_last_error(h)
        raise AtDnsError(rc, msg.decode() if msg else "")


def _ptr(arr, count=None, writable=False):
    """(pointer, where) of a float64 array: numpy (host) or CUDA torch tensor (device)."""
    if isinstance(arr, np.ndarray):
        if arr.dtype != np.float64 or not arr.flags["C_CONTIGUOUS"]:
            raise TypeError("host arrays must be C-contiguous float64")
        if writable and not arr.flags["WRITEABLE"]:
            raise TypeError("output array is read-only")
        if count is not None and arr.size < count:
            raise ValueError("array has %d elements, needs %d" % (arr.size, count))
        return arr.ctypes.data, AT_DNS_HOST
    mod = type(arr).__module__
    if mod.startswith("torch"):
        import torch
        if arr.dtype != torch.float64 or not arr.is_contiguous():
            raise TypeError("device tensors must be contiguous float64")
        if count is not None and arr.numel() < count:
            raise ValueError("tensor has %d elements, needs %d" % (arr.numel(), count))
        if arr.is_cuda:
            return arr.data_ptr(), AT_DNS_DEVICE
        return arr.data_ptr(), AT_DNS_HOST
    raise TypeError("expected a numpy array or a torch tensor")


def at_dns_config_default():
    cfg = at_dns_config_t()
    _check(load().at_dns_config_default(ctypes.byref(cfg)))
    return cfg


def at_dns_create(cfg):
    h = _P()
    _check(load().at_dns_create(ctypes.byref(cfg), ctypes.byref(h)))
    return h


def at_dns_set_state(h, u):
    p, where = _ptr(u)
    _check(load().at_dns_set_state(h, p, where), h)


def at_dns_set_history(h, levels, nlevels, step):
    p, where = _ptr(levels)
    _check(load().at_dns_set_history(h, p, nlevels, step, where), h)


def at_dns_get_state(h, out):
    p, where = _ptr(out, writable=True)
    _check(load().at_dns_get_state(h, p, where), h)


def at_dns_rhs(h, delay_mode, out):
    p, where = _ptr(out, writable=True)
    _check(load().at_dns_rhs(h, delay_mode, p, where), h)


def at_dns_step(h, nsteps, delay_mode):
    _check(load().at_dns_step(h, nsteps, delay_mode), h)


def at_dns_stats(h):
    s = at_dns_stats_t()
    _check(load().at_dns_stats(h, ctypes.byref(s)), h)
    return s


def at_dns_get_delay_map(h, step, mode, n_pes):
    out = np.zeros(n_pes * 6, dtype=np.uint8)
    _check(load().at_dns_get_delay_map(h, step, mode, out.ctypes.data), h)
    return out.reshape(n_pes, 6)


def at_dns_get_info(h):
    i = at_dns_info_t()
    _check(load().at_dns_get_info(h, ctypes.byref(i)), h)
    return i


def at_dns_profile(h, enable):
    _check(load().at_dns_profile(h, 1 if enable else 0), h)


def at_dns_kernel_times(h):
    arr = (at_dns_kernel_time_t * 16)()
    cnt = ctypes.c_int32(0)
    _check(load().at_dns_kernel_times(h, arr, 16, ctypes.byref(cnt)), h)
    return {arr[i].name.decode(): (int(arr[i].launches), float(arr[i].total_ms)) for i in range(cnt.value)}


def at_dns_set_kernel_path(h, path, tile=(0, 0, 0)):
    t = (ctypes.c_int32 * 3)(*[int(v) for v in tile])
    _check(load().at_dns_set_kernel_path(h, int(path), t), h)


def at_dns_synchronize(h):
    _check(load().at_dns_synchronize(h), h)


def at_dns_rhs_noalloc(n, gamma, prandtl, mu0, visc_exp, u_dev, rhs_dev, stream=None):
    """R(U) for one PE without device allocation (see include/at_dns.h): for
    callers that cannot allocate device memory.  u_dev and rhs_dev are CUDA
    float64 tensors of 5*n0*n1*n2 elements; the work is queued on `stream`."""
    cnt = 5 * int(n[0]) * int(n[1]) * int(n[2])
    pu, wu = _ptr(u_dev, cnt)
    pr, wr = _ptr(rhs_dev, cnt, writable=True)
    if wu != AT_DNS_DEVICE or wr != AT_DNS_DEVICE:
        raise TypeError("at_dns_rhs_noalloc takes device tensors")
    nn = (ctypes.c_int32 * 3)(*(int(v) for v in n))
    rc = load().at_dns_rhs_noalloc(nn, gamma, prandtl, mu0, visc_exp, pu, pr, stream)
    if rc != AT_DNS_OK:
        raise AtDnsError(rc, "at_dns_rhs_noalloc failed")


def at_dns_tune(h, delay_mode, trials=3):
    best = ctypes.c_double(0.0)
    _check(load().at_dns_tune(h, delay_mode, trials, ctypes.byref(best)), h)
    return best.value


def _bcheck(rc, b=None):
    if rc != AT_DNS_OK:
        msg = load().at_dns_batch_last_error(b)
        raise AtDnsError(rc, msg.decode() if msg else "")


def at_dns_batch_create(cfgs, stream=None):
    arr = (at_dns_config_t * len(cfgs))(*cfgs)
    b = _P()
    _bcheck(load().at_dns_batch_create(arr, len(cfgs), stream, ctypes.byref(b)))
    return b


def at_dns_batch_member(b, i):
    h = _P()
    _bcheck(load().at_dns_batch_member(b, i, ctypes.byref(h)), b)
    return h


def at_dns_batch_step(b, nsteps, delay_mode):
    _bcheck(load().at_dns_batch_step(b, nsteps, delay_mode), b)


def at_dns_batch_tune(b, delay_mode, trials=3):
    _bcheck(load().at_dns_batch_tune(b, delay_mode, trials), b)


def at_dns_wait_selftest(log2_polls=20):
    """Run the persistent step's bounded wait on a counter nothing advances;
    True when it gave up (the expected result)."""
    out = ctypes.c_int32(-1)
    _check(load().at_dns_wait_selftest(log2_polls, ctypes.byref(out)))
    return out.value == 1


def _byte_ptr(buf, size):
    """(pointer, where) of a byte buffer of at least `size` bytes: a numpy
    uint8 array (host) or a uint8 torch tensor (host or CUDA)."""
    if isinstance(buf, np.ndarray):
        if buf.dtype != np.uint8 or not buf.flags["C_CONTIGUOUS"] or buf.size < size:
            raise TypeError("checkpoint buffers are C-contiguous uint8 arrays of at least %d bytes" % size)
        return buf.ctypes.data, AT_DNS_HOST
    if type(buf).__module__.startswith("torch"):
        import torch
        if buf.dtype != torch.uint8 or not buf.is_contiguous() or buf.numel() < size:
            raise TypeError("checkpoint buffers are contiguous uint8 tensors of at least %d bytes" % size)
        return buf.data_ptr(), (AT_DNS_DEVICE if buf.is_cuda else AT_DNS_HOST)
    raise TypeError("expected a numpy array or a torch tensor")


def at_dns_checkpoint_size(h):
    n = ctypes.c_int64(0)
    _check(load().at_dns_checkpoint_size(h, ctypes.byref(n)), h)
    return int(n.value)


def at_dns_checkpoint_save(h, buf):
    p, where = _byte_ptr(buf, at_dns_checkpoint_size(h))
    _check(load().at_dns_checkpoint_save(h, p, where), h)


def at_dns_checkpoint_load(h, buf):
    p, where = _byte_ptr(buf, 0)
    _check(load().at_dns_checkpoint_load(h, p, where), h)


def at_dns_batch_destroy(b):
    load().at_dns_batch_destroy(b)


def at_dns_last_error(h=None):
    m = load().at_dns_last_error(h)
    return m.decode() if m else ""


def at_dns_destroy(h):
    load().at_dns_destroy(h)


def make_config(n=(32, 32, 32), pes=(1, 1, 1), precision="p64", stream=None, path="auto", **kw):
    cfg = at_dns_config_default()
    cfg.kernel_path = PATHS[path] if isinstance(path, str) else int(path)
    for d in range(3):
        cfg.n[d] = int(n[d])
        cfg.pes[d] = int(pes[d])
    cfg.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    if stream is not None:
        cfg.stream = stream
    pool = kw.pop("pool", None)
    if pool is not None:
        if hasattr(pool, "data_ptr"):        # a device tensor lends its memory
            cfg.pool = pool.data_ptr()
            cfg.pool_bytes = pool.numel() * pool.element_size()
        else:
            cfg.pool = int(pool)
    for k, v in kw.items():
        if not hasattr(cfg, k):
            raise TypeError("unknown configuration field %r" % k)
        setattr(cfg, k, v)
    return cfg


class Batch:
    """Independent members advancing together: one graph launch per step (each
    member on its own branch), or, opted into with set_persistent(True) when
    every member is eligible (at most 64 members, FP32 forms, 4th order, AB2,
    unforced, PE extents fitting one paired tile), one persistent kernel
    launch per step.  `members` is a list of dicts of Solver arguments (n,
    pes, precision, ...); `persistent` sets the step form at creation."""

    def __init__(self, members, stream=None, persistent=False):
        self.specs = [dict(m) for m in members]
        cfgs = [make_config(**m) for m in self.specs]
        self.b = at_dns_batch_create(cfgs, stream)
        self.members = []
        for i, m in enumerate(self.specs):
            h = at_dns_batch_member(self.b, i)
            self.members.append(Solver(n=m.get("n", (32, 32, 32)), pes=m.get("pes", (1, 1, 1)), handle=h))
        if persistent:
            self.set_persistent(True)

    def __len__(self):
        return len(self.members)

    def __getitem__(self, i):
        return self.members[i]

    def step(self, nsteps=1, mode="sync"):
        at_dns_batch_step(self.b, nsteps, MODES.get(mode, mode))

    def tune(self, mode="random", trials=3):
        at_dns_batch_tune(self.b, MODES.get(mode, mode), trials)

    def set_persistent(self, enable=True):
        """Allow or forbid the persistent single-launch step; returns whether
        the next step uses it."""
        out = ctypes.c_int32(0)
        _bcheck(load().at_dns_batch_persistent(self.b, 1 if enable else 0, ctypes.byref(out)), self.b)
        return bool(out.value)

    @property
    def persistent(self):
        """Whether the next step runs as one persistent kernel launch."""
        out = ctypes.c_int32(0)
        _bcheck(load().at_dns_batch_persistent(self.b, -1, ctypes.byref(out)), self.b)
        return bool(out.value)

    def close(self):
        if self.b:
            for m in self.members:
                m.h = None
            at_dns_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Solver:
    """Owns one handle; methods map one-to-one onto the C ABI."""

    def __init__(self, n=(32, 32, 32), pes=(1, 1, 1), precision="p64", stream=None, path="auto", handle=None,
                 **kw):
        self._pool = kw.get("pool")            # kept alive as long as the handle
        cfg = make_config(n, pes, precision, stream, path, **kw)
        self.cfg = cfg
        self.n = tuple(int(v) for v in n)
        self.pes = tuple(int(v) for v in pes)
        self.npts = self.n[0] * self.n[1] * self.n[2]
        self._owned = handle is None
        self.h = at_dns_create(cfg) if handle is None else handle

    @property
    def n_pes(self):
        return self.pes[0] * self.pes[1] * self.pes[2]

    def set_state(self, u):
        at_dns_set_state(self.h, u)

    def set_history(self, levels, step):
        """levels: list of fields [U^step, U^(step-1), ...] or an array shaped
        (nlevels, 5, nz, ny, nx)."""
        if isinstance(levels, (list, tuple)):
            levels = np.ascontiguousarray(np.stack(levels))
        if len(levels.shape) != 5:
            raise ValueError("levels must be shaped (nlevels, 5, nz, ny, nx)")
        at_dns_set_history(self.h, levels, int(levels.shape[0]), step)

    def get_state(self, out=None):
        if out is None:
            out = np.empty((5, self.n[2], self.n[1], self.n[0]))
        at_dns_get_state(self.h, out)
        return out

    def rhs(self, mode="sync", out=None):
        if out is None:
            out = np.empty((5, self.n[2], self.n[1], self.n[0]))
        at_dns_rhs(self.h, MODES.get(mode, mode), out)
        return out

    def step(self, nsteps=1, mode="sync"):
        at_dns_step(self.h, nsteps, MODES.get(mode, mode))

    def stats(self):
        return at_dns_stats(self.h).as_dict()

    def delay_map(self, step, mode="random"):
        return at_dns_get_delay_map(self.h, step, MODES.get(mode, mode), self.n_pes)

    def info(self):
        i = at_dns_get_info(self.h)
        out = {name: getattr(i, name) for name, _ in i._fields_}
        out["tile"] = list(i.tile)
        return out

    def checkpoint(self, out=None):
        """The run state as a checkpoint buffer (a new host uint8 array, or
        `out`: a uint8 numpy array or torch tensor, host or CUDA)."""
        if out is None:
            out = np.empty(at_dns_checkpoint_size(self.h), dtype=np.uint8)
        at_dns_checkpoint_save(self.h, out)
        return out

    def restore(self, buf):
        """Continue the run saved in `buf` (same configuration)."""
        at_dns_checkpoint_load(self.h, buf)

    def synchronize(self):
        at_dns_synchronize(self.h)

    def profile(self, enable=True):
        at_dns_profile(self.h, enable)

    def kernel_times(self):
        return at_dns_kernel_times(self.h)

    def set_kernel_path(self, path, tile=(0, 0, 0)):
        at_dns_set_kernel_path(self.h, PATHS[path] if isinstance(path, str) else int(path), tile)

    def tune(self, mode="random", trials=3):
        return at_dns_tune(self.h, MODES.get(mode, mode), trials)

    def close(self):
        if self.h and self._owned:
            at_dns_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
