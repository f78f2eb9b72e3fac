"""Python binding of the C ABI in include/rad.h (argument marshalling only).

Every computation runs in the CUDA library librad.so; this module converts
arguments (torch tensors / numpy arrays -> pointers, torch streams -> cudaStream_t)
and raises on non-OK statuses.  There is no CPU fallback: if the library is not
built or cannot be loaded, every entry point raises RuntimeError.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# The library the binding loads: librad.so, or another build of it (such as
# librad_debug.so, with the kernels' index checks) named by RAD_LIBRARY.
LIB_PATH = os.environ.get("RAD_LIBRARY") or os.path.join(_HERE, "librad.so")

RAD_OK, RAD_EINVAL, RAD_ENOMEM, RAD_ECUDA, RAD_EDATA, RAD_ETIMEOUT, RAD_EBUSY, RAD_ESTATE = range(8)
FF_POINT, FF_CIC, FF_TSC, FF_QSC, FF_GAUSS = range(5)
FF_3D = 1  # rad_ff.flags: box shapes as axis-aligned 3-D products
PREC_MIXED, PREC_FP64 = 0, 1
STATUS_NAMES = ["RAD_OK", "RAD_EINVAL", "RAD_ENOMEM", "RAD_ECUDA", "RAD_EDATA", "RAD_ETIMEOUT",
                "RAD_EBUSY", "RAD_ESTATE"]

# Every symbol include/rad.h and include/rad_probe.h declare.
EXPORTS = [
    "rad_create", "rad_accumulate", "rad_spectrum", "rad_spectrum_ff", "rad_spectrum_species",
    "rad_sync", "rad_reset",
    "rad_destroy", "rad_state_size", "rad_state_export", "rad_state_import", "rad_state_merge",
    "rad_get_tile", "rad_set_tile", "rad_tune", "rad_batch_create", "rad_batch_accumulate",
    "rad_batch_sync", "rad_batch_destroy", "rad_server_create", "rad_server_set_policy", "rad_job_submit", "rad_job_feed",
    "rad_job_finish", "rad_job_poll", "rad_job_result", "rad_server_stats_get",
    "rad_server_destroy", "rad_status_str", "rad_last_error", "rad_kernel_launch_count",
    "rad_probe_peaks", "rad_probe_tensor", "rad_probe_loop", "rad_profile_enable", "rad_profile_read", "rad_profile_clock", "rad_accumulate_static",
    "rad_static_status",
    "rad_spectrum_literal", "rad_push_step", "rad_push_flush",
    "rad_selftest_wait", "rad_selftest_stage1", "rad_selftest_phase",
]
FF_LITERAL = 2  # rad_ff.flags at creation: also accumulate the paper's literal sum
# Round policies of the serving loop (rad_server_set_policy).
SERVE_ALL, SERVE_OLDEST, SERVE_LEAST_SERVED, SERVE_LEAST_SERVED_AGED = 0, 1, 2, 3
SERVE_OLDEST_BACKFILL = 4

# Limits of rad_accumulate_static (include/rad.h).
STATIC_MAX_OMEGA, STATIC_MAX_DIRS, STATIC_MAX_BINS, STATIC_MAX_PARTICLES = 4096, 4096, 65536, 65536


class RadError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{where}: {name}")


class rad_ff(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("flags", ctypes.c_int32), ("width", ctypes.c_double)]


class rad_tile(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int32), ("omega_tile", ctypes.c_int32),
                ("chunk", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class rad_step(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("r", ctypes.c_void_p), ("beta", ctypes.c_void_p),
                ("beta_dot", ctypes.c_void_p), ("w", ctypes.c_void_p), ("t", ctypes.c_double),
                ("dt", ctypes.c_double)]


class rad_job_desc(ctypes.Structure):
    _fields_ = [("omega", ctypes.c_void_p), ("n_omega", ctypes.c_int32), ("n_dir", ctypes.c_int32),
                ("dirs", ctypes.c_void_p), ("ff", rad_ff), ("max_particles", ctypes.c_int64),
                ("max_queued", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class rad_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("admitted", ctypes.c_int64),
                ("completed", ctypes.c_int64), ("rounds", ctypes.c_int64),
                ("updates", ctypes.c_int64), ("footprint_bytes", ctypes.c_int64),
                ("peak_footprint_bytes", ctypes.c_int64), ("active", ctypes.c_int32),
                ("waiting", ctypes.c_int32)]


_lib = None


def load(path: str = LIB_PATH):
    """Load librad.so (raises RuntimeError if it is missing or broken)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} is missing (run the package build)")
    lib = ctypes.CDLL(path)
    vp, i32, i64, dbl, st = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_int
    sig = {
        "rad_create": (st, [vp, i32, vp, i32, rad_ff, i32, vp, ctypes.POINTER(vp)]),
        "rad_accumulate": (st, [vp, i64, vp, vp, vp, vp, dbl, dbl]),
        "rad_spectrum": (st, [vp, vp, vp, vp]),
        "rad_spectrum_ff": (st, [vp, rad_ff, vp, vp, vp]),
        "rad_spectrum_species": (st, [vp, vp, i32, vp, vp, vp]),
        "rad_sync": (st, [vp]),
        "rad_reset": (st, [vp]),
        "rad_destroy": (None, [vp]),
        "rad_state_size": (ctypes.c_size_t, [vp]),
        "rad_state_export": (st, [vp, vp, ctypes.c_size_t]),
        "rad_state_import": (st, [vp, vp, ctypes.c_size_t]),
        "rad_state_merge": (st, [vp, vp, ctypes.c_size_t]),
        "rad_get_tile": (st, [vp, ctypes.POINTER(rad_tile)]),
        "rad_set_tile": (st, [vp, ctypes.POINTER(rad_tile)]),
        "rad_tune": (st, [vp, i64]),
        "rad_batch_create": (st, [ctypes.POINTER(vp), i32, vp, ctypes.POINTER(vp)]),
        "rad_batch_accumulate": (st, [vp, ctypes.POINTER(rad_step)]),
        "rad_batch_sync": (st, [vp]),
        "rad_batch_destroy": (None, [vp]),
        "rad_server_create": (st, [ctypes.c_size_t, i32, vp, ctypes.POINTER(vp)]),
        "rad_server_set_policy": (st, [vp, i32, i64]),
        "rad_job_submit": (st, [vp, ctypes.POINTER(rad_job_desc), ctypes.POINTER(i64)]),
        "rad_job_feed": (st, [vp, i64, ctypes.POINTER(rad_step)]),
        "rad_job_finish": (st, [vp, i64]),
        "rad_job_poll": (st, [vp, i64, ctypes.POINTER(i32)]),
        "rad_job_result": (st, [vp, i64, dbl, vp, vp, vp, ctypes.POINTER(dbl)]),
        "rad_server_stats_get": (st, [vp, ctypes.POINTER(rad_server_stats)]),
        "rad_server_destroy": (None, [vp]),
        "rad_status_str": (ctypes.c_char_p, [st]),
        "rad_last_error": (st, [vp]),
        "rad_kernel_launch_count": (i64, []),
        "rad_probe_peaks": (ctypes.c_int, [vp, ctypes.c_int]),
        "rad_probe_tensor": (ctypes.c_int, [vp, ctypes.c_int]),
        "rad_probe_loop": (ctypes.c_int, [vp, ctypes.c_int]),
        "rad_profile_enable": (st, [vp, i32]),
        "rad_profile_read": (st, [vp, ctypes.POINTER(dbl), ctypes.POINTER(dbl), ctypes.POINTER(i64)]),
        "rad_profile_clock": (st, [vp, ctypes.POINTER(dbl)]),
        "rad_selftest_wait": (st, [i64, ctypes.POINTER(i32), ctypes.POINTER(dbl)]),
        "rad_selftest_stage1": (st, [vp, i64, vp, vp, vp, vp, dbl, dbl, i32, vp, vp]),
        "rad_selftest_phase": (st, [vp, i32, vp, vp, vp, vp]),
        "rad_accumulate_static": (st, [vp, i32, vp, i32, i64, vp, vp, vp, vp, dbl, dbl, vp, vp]),
        "rad_static_status": (st, [vp]),
        "rad_spectrum_literal": (st, [vp, vp]),
        "rad_push_step": (st, [vp, i64, vp, vp, vp, dbl, dbl]),
        "rad_push_flush": (st, [vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(status: int, where: str) -> None:
    if status != RAD_OK:
        raise RadError(status, where)


def _ptr(x) -> int:
    """Address of a torch tensor / numpy array (must be contiguous float64 where it matters)."""
    if x is None:
        return 0
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        if not x.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    raise TypeError(f"unsupported buffer type {type(x)}")


def _f64_host(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _stream_handle(stream) -> int:
    if stream is None:
        return 0
    if hasattr(stream, "cuda_stream"):
        return int(stream.cuda_stream)
    return int(stream)


def _check_particles(n, *arrs):
    for a in arrs:
        if hasattr(a, "dtype") and str(a.dtype) not in ("torch.float64", "float64"):
            raise TypeError("particle arrays must be float64")


def kernel_launch_count() -> int:
    return int(load().rad_kernel_launch_count())


def probe_peaks() -> np.ndarray:
    out = np.zeros(16)
    rc = load().rad_probe_peaks(out.ctypes.data, 16)
    if rc != 0:
        raise RuntimeError(f"rad_probe_peaks failed with CUDA error {rc}")
    return out


def selftest_wait(limit_ns: int) -> tuple:
    """rad_selftest_wait: (timed_out, waited_s) of a bounded wait nothing completes."""
    flag, waited = ctypes.c_int32(), ctypes.c_double()
    _check(load().rad_selftest_wait(int(limit_ns), ctypes.byref(flag), ctypes.byref(waited)),
           "rad_selftest_wait")
    return bool(flag.value), waited.value


def spectrum_species(contexts, ffs, out=None, accept_edata: bool = False):
    """rad_spectrum_species: (coherent, incoherent, total) of several species, each a
    Context on the same grid with its own shape ffs[s] = (kind, width[, flags]);
    the coherent amplitudes of all species add before |.|^2."""
    contexts = list(contexts)
    n = len(contexts)
    if n != len(ffs):
        raise ValueError("one shape per species")
    c0 = contexts[0]
    if out is None:
        out = tuple(np.zeros((c0.n_dir, c0.n_omega)) for _ in range(3))
    handles = (ctypes.c_void_p * n)(*[c.handle.value for c in contexts])
    shapes = (rad_ff * n)(*[rad_ff(int(f[0]), int(f[2]) if len(f) > 2 else 0, float(f[1])) for f in ffs])
    st = load().rad_spectrum_species(ctypes.addressof(handles), ctypes.addressof(shapes), n,
                                     *[_ptr(o) for o in out])
    if not (accept_edata and st == RAD_EDATA):
        _check(st, "rad_spectrum_species")
    return out


def probe_tensor() -> np.ndarray:
    """rad_probe_tensor: [mma.sync TF32 MACs/clk/SM, clocks per tcgen05.mma kind::tf32 at
    N = 16, 64, 128, 256, kind::f16 at N = 16, 256, probe MHz]."""
    out = np.zeros(8)
    rc = load().rad_probe_tensor(out.ctypes.data, 8)
    if rc != 0:
        raise RuntimeError(f"rad_probe_tensor failed with CUDA error {rc}")
    return out


def probe_loop() -> np.ndarray:
    """rad_probe_loop: [MUFU lane-ops/clk/SM, MHz] for the update loop as it is (0),
    without the TF32 split (1), without the MMAs (2), without either (3), and the
    variant-9 loop (4)."""
    out = np.zeros(10)
    rc = load().rad_probe_loop(out.ctypes.data, 10)
    if rc != 0:
        raise RuntimeError(f"rad_probe_loop failed with CUDA error {rc}")
    return out


class Context:
    """One spectrum job: rad_create / rad_accumulate / rad_spectrum."""

    def __init__(self, omega, dirs, ff_kind: int = FF_POINT, ff_width: float = 0.0,
                 prec: int = PREC_MIXED, stream=None, ff_flags: int = 0):
        lib = load()
        self._ff_flags = int(ff_flags)
        self.omega = _f64_host(omega).ravel()
        self.dirs = _f64_host(dirs).reshape(-1, 3)
        self.n_omega, self.n_dir = self.omega.shape[0], self.dirs.shape[0]
        h = ctypes.c_void_p()
        _check(lib.rad_create(self.omega.ctypes.data, self.n_omega, self.dirs.ctypes.data,
                              self.n_dir, rad_ff(ff_kind, self._ff_flags, ff_width), prec,
                              _stream_handle(stream), ctypes.byref(h)), "rad_create")
        self._h = h
        self._lib = lib

    @property
    def handle(self):
        return self._h

    def close(self) -> None:
        if getattr(self, "_h", None) and self._h.value:
            self._lib.rad_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def accumulate(self, r, beta, beta_dot, w, t: float, dt: float) -> None:
        """Add one time step; r, beta, beta_dot are [3][N] and w [N], float64,
        torch CUDA tensors or host arrays."""
        n = int(w.shape[0])
        _check_particles(n, r, beta, beta_dot, w)
        _check(self._lib.rad_accumulate(self._h, n, _ptr(r), _ptr(beta), _ptr(beta_dot), _ptr(w),
                                        float(t), float(dt)), "rad_accumulate")

    def spectrum(self, ff: Optional[tuple] = None, out=None):
        """Return (coherent, incoherent, total) as [n_dir][n_omega] arrays.

        out: optional tuple of three preallocated float64 buffers (torch CUDA
        tensors or numpy arrays); otherwise numpy arrays are returned."""
        if out is None:
            out = tuple(np.zeros((self.n_dir, self.n_omega)) for _ in range(3))
        ptrs = [_ptr(o) for o in out]
        if ff is None:
            st = self._lib.rad_spectrum(self._h, *ptrs)
        else:
            flags = int(ff[2]) if len(ff) > 2 else 0
            st = self._lib.rad_spectrum_ff(self._h, rad_ff(int(ff[0]), flags, float(ff[1])), *ptrs)
        _check(st, "rad_spectrum")
        return out

    def push_step(self, r, beta, w, t: float, dt: float) -> None:
        """In-situ coupling: hand over one step without beta_dot (finite differences
        of consecutive steps on the device; see rad_push_step)."""
        n = int(w.shape[0])
        _check_particles(n, r, beta, w)
        _check(self._lib.rad_push_step(self._h, n, _ptr(r), _ptr(beta), _ptr(w), float(t), float(dt)),
               "rad_push_step")

    def push_flush(self) -> None:
        _check(self._lib.rad_push_flush(self._h), "rad_push_flush")

    def spectrum_literal(self, out=None):
        """The paper's literal spectrum K0 |P|^2 (contexts created with FF_LITERAL)."""
        if out is None:
            out = np.zeros((self.n_dir, self.n_omega))
        _check(self._lib.rad_spectrum_literal(self._h, _ptr(out)), "rad_spectrum_literal")
        return out

    def sync(self) -> None:
        _check(self._lib.rad_sync(self._h), "rad_sync")

    def reset(self) -> None:
        _check(self._lib.rad_reset(self._h), "rad_reset")

    def state_export(self) -> bytes:
        n = self._lib.rad_state_size(self._h)
        buf = ctypes.create_string_buffer(n)
        _check(self._lib.rad_state_export(self._h, buf, n), "rad_state_export")
        return buf.raw

    def state_import(self, blob: bytes) -> None:
        _check(self._lib.rad_state_import(self._h, blob, len(blob)), "rad_state_import")

    def state_merge(self, blob: bytes) -> None:
        _check(self._lib.rad_state_merge(self._h, blob, len(blob)), "rad_state_merge")

    def get_tile(self) -> tuple:
        t = rad_tile()
        _check(self._lib.rad_get_tile(self._h, ctypes.byref(t)), "rad_get_tile")
        return (t.variant, t.omega_tile, t.chunk)

    def set_tile(self, variant: int, omega_tile: int = 0, chunk: int = 0) -> None:
        t = rad_tile(variant, omega_tile, chunk, 0)
        _check(self._lib.rad_set_tile(self._h, ctypes.byref(t)), "rad_set_tile")

    def tune(self, n: int) -> tuple:
        _check(self._lib.rad_tune(self._h, int(n)), "rad_tune")
        return self.get_tile()

    def last_error(self) -> int:
        return int(self._lib.rad_last_error(self._h))

    def profile(self, on: bool = True) -> None:
        _check(self._lib.rad_profile_enable(self._h, 1 if on else 0), "rad_profile_enable")

    def profile_read(self) -> tuple:
        """(prepass_ms, accumulate_ms, calls) summed since the last read."""
        a, b, n = ctypes.c_double(), ctypes.c_double(), ctypes.c_int64()
        _check(self._lib.rad_profile_read(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(n)),
               "rad_profile_read")
        return a.value, b.value, n.value

    def selftest_stage1(self, r, beta, beta_dot, w, t: float, dt: float, direction: int):
        """rad_selftest_stage1: per particle (th, tl, a0..a3, fast, 0) for one direction
        (device arrays) and the direction's transverse basis (e1, e2)."""
        n = int(w.shape[0])
        out = np.zeros((n, 8), dtype=np.float32)
        basis = np.zeros(6, dtype=np.float32)
        _check(self._lib.rad_selftest_stage1(self._h, n, _ptr(r), _ptr(beta), _ptr(beta_dot), _ptr(w),
                                             float(t), float(dt), int(direction), out.ctypes.data,
                                             basis.ctypes.data), "rad_selftest_stage1")
        return out, basis.reshape(2, 3)

    def selftest_phase(self, th, tl):
        """rad_selftest_phase: (fast, wide) phases in radians, [n_omega][len(th)]."""
        th = np.ascontiguousarray(th, dtype=np.float32)
        tl = np.ascontiguousarray(tl, dtype=np.float32)
        fast = np.zeros((self.n_omega, th.shape[0]), dtype=np.float32)
        wide = np.zeros_like(fast)
        _check(self._lib.rad_selftest_phase(self._h, th.shape[0], th.ctypes.data, tl.ctypes.data,
                                            fast.ctypes.data, wide.ctypes.data), "rad_selftest_phase")
        return fast, wide

    def profile_clock(self) -> float:
        """Effective SM clock (MHz) of the accumulate kernels since the last call."""
        m = ctypes.c_double()
        _check(self._lib.rad_profile_clock(self._h, ctypes.byref(m)), "rad_profile_clock")
        return m.value


def accumulate_static(omega, dirs, r, beta, beta_dot, w, t: float, dt: float, state,
                      stream=None) -> None:
    """rad_accumulate_static: one step into caller-owned accumulators `state`
    (device float32 [16][n_omega * n_dir]) with no allocation by the library.
    omega [n_omega], dirs [n_dir][3] and the particle arrays are float64 device
    tensors; see include/rad.h for the limits."""
    n = int(w.shape[0])
    _check_particles(n, r, beta, beta_dot, w)
    n_omega = int(omega.shape[0])
    n_dir = int(dirs.numel() // 3) if hasattr(dirs, "numel") else int(np.asarray(dirs).size // 3)
    _check(load().rad_accumulate_static(_ptr(omega), n_omega, _ptr(dirs), n_dir, n, _ptr(r),
                                        _ptr(beta), _ptr(beta_dot), _ptr(w), float(t), float(dt),
                                        _ptr(state), _stream_handle(stream)),
           "rad_accumulate_static")


def static_status(stream=None) -> int:
    """rad_static_status: the device's report on the latest accumulate_static call
    on the current device, as a status code (RAD_OK, RAD_EDATA, RAD_EINVAL,
    RAD_ETIMEOUT, RAD_ECUDA); synchronises the stream."""
    return int(load().rad_static_status(_stream_handle(stream)))


def make_step(n, r, beta, beta_dot, w, t, dt) -> rad_step:
    """A rad_step pointing at the four arrays (float64, contiguous; host or device).  The
    step keeps references to them, so they stay alive as long as the step does."""
    _check_particles(int(n), r, beta, beta_dot, w)
    st = rad_step(int(n), _ptr(r), _ptr(beta), _ptr(beta_dot), _ptr(w), float(t), float(dt))
    st._keep = (r, beta, beta_dot, w)
    return st


class Batch:
    """Many contexts advanced together in one persistent launch per step."""

    def __init__(self, contexts: Sequence[Context], stream=None):
        lib = load()
        self.contexts = list(contexts)
        arr = (ctypes.c_void_p * len(self.contexts))(*[c.handle.value for c in self.contexts])
        h = ctypes.c_void_p()
        _check(lib.rad_batch_create(arr, len(self.contexts), _stream_handle(stream),
                                    ctypes.byref(h)), "rad_batch_create")
        self._h, self._lib = h, lib

    def accumulate(self, steps: Sequence[rad_step]) -> None:
        arr = (rad_step * len(steps))(*steps)
        _check(self._lib.rad_batch_accumulate(self._h, arr), "rad_batch_accumulate")

    def sync(self) -> None:
        _check(self._lib.rad_batch_sync(self._h), "rad_batch_sync")

    def close(self) -> None:
        if getattr(self, "_h", None) and self._h.value:
            self._lib.rad_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching request loop (rad_server_*)."""

    def __init__(self, hbm_budget: int, max_slots: int, stream=None):
        lib = load()
        h = ctypes.c_void_p()
        _check(lib.rad_server_create(int(hbm_budget), int(max_slots), _stream_handle(stream),
                                     ctypes.byref(h)), "rad_server_create")
        self._h, self._lib = h, lib

    def set_policy(self, policy: int, round_updates: int = 0) -> None:
        """rad_server_set_policy: SERVE_ALL, SERVE_OLDEST, SERVE_LEAST_SERVED or SERVE_LEAST_SERVED_AGED."""
        _check(self._lib.rad_server_set_policy(self._h, int(policy), int(round_updates)),
               "rad_server_set_policy")

    def submit(self, omega, dirs, ff_kind=FF_POINT, ff_width=0.0, max_particles=1,
               max_queued=2) -> int:
        om = _f64_host(omega).ravel()
        di = _f64_host(dirs).reshape(-1, 3)
        d = rad_job_desc(om.ctypes.data, om.shape[0], di.shape[0], di.ctypes.data,
                         rad_ff(ff_kind, 0, ff_width), int(max_particles), int(max_queued), 0)
        jid = ctypes.c_int64()
        _check(self._lib.rad_job_submit(self._h, ctypes.byref(d), ctypes.byref(jid)), "rad_job_submit")
        return jid.value

    def feed(self, job: int, step: rad_step) -> int:
        """Returns the status (RAD_OK or RAD_EBUSY); raises on other errors."""
        st = self._lib.rad_job_feed(self._h, int(job), ctypes.byref(step))
        if st not in (RAD_OK, RAD_EBUSY):
            raise RadError(st, "rad_job_feed")
        return st

    def finish(self, job: int) -> None:
        _check(self._lib.rad_job_finish(self._h, int(job)), "rad_job_finish")

    def poll(self, job: int) -> bool:
        d = ctypes.c_int32()
        _check(self._lib.rad_job_poll(self._h, int(job), ctypes.byref(d)), "rad_job_poll")
        return bool(d.value)

    def result(self, job: int, n_dir: int, n_omega: int, timeout: float = -1.0,
               accept_edata: bool = False):
        """(coherent, incoherent, total, latency_s).  A job that saw invalid particles
        (RAD_EDATA) raises unless accept_edata; its spectrum then covers the valid ones."""
        outs = [np.zeros((n_dir, n_omega)) for _ in range(3)]
        lat = ctypes.c_double()
        st = self._lib.rad_job_result(self._h, int(job), float(timeout), *[o.ctypes.data for o in outs],
                                      ctypes.byref(lat))
        if not (accept_edata and st == RAD_EDATA):
            _check(st, "rad_job_result")
        return outs[0], outs[1], outs[2], lat.value

    def stats(self) -> dict:
        s = rad_server_stats()
        _check(self._lib.rad_server_stats_get(self._h, ctypes.byref(s)), "rad_server_stats_get")
        return {f: getattr(s, f) for f, _ in rad_server_stats._fields_}

    def close(self) -> None:
        if getattr(self, "_h", None) and self._h.value:
            self._lib.rad_server_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
