"""FP64 CPU oracle for the Lienard-Wiechert radiation sum with form factors.

TEST INFRASTRUCTURE ONLY: the slow, plain definition (``rad_oracle.c``) that
the CUDA library is checked against.  Only the test suite, the smoke check and
the benchmark's CPU-baseline leg may import this package; the library itself
never does.  It shares no code with the CUDA path.

What is computed is documented in ``rad_oracle.c``: per accumulate call and per
(direction, frequency) bin, the coherent sum U (weights w dt), the incoherent
sum V (weights sqrt(w) dt) and the paper's literal sum P (weights F_k dt) of
A_k exp(i omega (t - n.r_k/c)) (Eq. 1, Eq. 13), read out as
I_coh = K0 f^2 |U|^2, I_inc = K0 (1-f^2) |V|^2, I_tot = I_coh + I_inc and
I_paper = K0 |P|^2, with f the normalised amplitude form factor of Table 1.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rad_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

FF_POINT, FF_CIC, FF_TSC, FF_QSC, FF_GAUSS = 0, 1, 2, 3, 4
FF_3D = 1  # ff_flags bit: box shapes as axis-aligned 3-D products (direction-dependent f)
PER_BIN = 18  # U, V, P: complex 3-vectors

_lib = None


def build(force: bool = False) -> str:
    """Compile rad_oracle.c into liboracle.so (OpenMP when gcc supports it)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    base = ["gcc", "-O2", "-shared", "-fPIC", "-std=c11", "-o", _LIB, _SRC, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    dp = ctypes.POINTER(ctypes.c_double)
    i64 = ctypes.c_int64
    lib.oracle_k0.restype = ctypes.c_double
    lib.oracle_form_factor.restype = ctypes.c_double
    lib.oracle_form_factor.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double]
    lib.oracle_form_factor_dir.restype = ctypes.c_double
    lib.oracle_form_factor_dir.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                           ctypes.c_double, dp]
    lib.oracle_amplitude.argtypes = [dp, dp, dp, dp]
    lib.oracle_accumulate.argtypes = [i64, dp, dp, i64, dp, dp, dp, dp, ctypes.c_double,
                                      ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                      ctypes.c_double, dp, dp]
    lib.oracle_accumulate_particles.argtypes = [i64, dp, dp, i64, dp, dp, dp, ctypes.c_double,
                                                ctypes.c_double, dp]
    lib.oracle_readout.argtypes = [i64, dp, dp, dp, dp, ctypes.c_int, ctypes.c_int,
                                   ctypes.c_double, dp, dp, dp, dp]
    lib.oracle_num_threads.restype = ctypes.c_int
    _lib = lib
    return lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def k0() -> float:
    """q_e^2 / (16 pi^3 eps0 c), the prefactor of Eq. 1."""
    return _load().oracle_k0()


def num_threads() -> int:
    return _load().oracle_num_threads()


def form_factor(kind: int, width: float, omega) -> np.ndarray:
    """Normalised amplitude form factor f(omega) of Table 1 (f(0) = 1)."""
    lib = _load()
    om = np.atleast_1d(_f64(omega))
    return np.array([lib.oracle_form_factor(int(kind), float(width), float(w)) for w in om])


def form_factor_dir(kind: int, flags: int, width: float, omega: float, n) -> float:
    """f(n, omega): Table 1, or with FF_3D the axis-aligned 3-D product of the box shape."""
    n = _f64(n)
    return _load().oracle_form_factor_dir(int(kind), int(flags), float(width), float(omega), _p(n))


def amplitude(n, beta, bdot) -> np.ndarray:
    """A = n x [(n - beta) x betadot] / (1 - beta.n)^2 (Eq. 1) for one particle."""
    n, beta, bdot = _f64(n), _f64(beta), _f64(bdot)
    out = np.zeros(3)
    _load().oracle_amplitude(_p(n), _p(beta), _p(bdot), _p(out))
    return out


def grid_bins(omega, dirs, bins=None):
    """Per-bin (omega, n) arrays for a direction x frequency grid.

    bins: None for the full grid in row-major [n_dir][n_omega] order, else an
    iterable of (i_dir, i_omega) pairs.
    """
    omega = _f64(omega)
    dirs = _f64(dirs).reshape(-1, 3)
    if bins is None:
        bo = np.tile(omega, dirs.shape[0])
        bd = np.repeat(dirs, omega.shape[0], axis=0)
    else:
        bins = np.asarray(list(bins), dtype=np.int64).reshape(-1, 2)
        bo = omega[bins[:, 1]]
        bd = dirs[bins[:, 0]]
    return _f64(bo), _f64(bd)


class Accumulator:
    """Running oracle sums over a set of bins (Eq. 13, split and literal)."""

    def __init__(self, bin_omega, bin_dir, ff_kind: int = FF_POINT, ff_width: float = 0.0,
                 ff_flags: int = 0):
        self.bin_omega = _f64(bin_omega).ravel()
        self.bin_dir = _f64(bin_dir).reshape(-1, 3)
        assert self.bin_dir.shape[0] == self.bin_omega.shape[0]
        self.ff_kind, self.ff_width, self.ff_flags = int(ff_kind), float(ff_width), int(ff_flags)
        nb = self.bin_omega.shape[0]
        self.acc = np.zeros((nb, PER_BIN))
        self.comp = np.zeros((nb, PER_BIN))

    @property
    def n_bins(self) -> int:
        return self.bin_omega.shape[0]

    def accumulate(self, r, beta, beta_dot, w, t: float, dt: float) -> None:
        """Add one call's particles; r, beta, beta_dot are SoA [3][N], w is [N]."""
        r, beta, bd, w = _f64(r), _f64(beta), _f64(beta_dot), _f64(w)
        N = w.shape[0]
        assert r.size == 3 * N and beta.size == 3 * N and bd.size == 3 * N
        _load().oracle_accumulate(self.n_bins, _p(self.bin_omega), _p(self.bin_dir), N, _p(r),
                                  _p(beta), _p(bd), _p(w), float(t), float(dt), self.ff_kind,
                                  self.ff_flags, self.ff_width, _p(self.acc), _p(self.comp))

    def amplitudes(self) -> dict:
        """Compensated complex sums: U, V, P as [n_bins][3] complex arrays."""
        s = self.acc + self.comp
        z = s[:, 0::2] + 1j * s[:, 1::2]  # [nb][9]: U xyz, V xyz, P xyz
        return {"U": z[:, 0:3], "V": z[:, 3:6], "P": z[:, 6:9]}

    def spectra(self, ff_kind: int | None = None, ff_width: float | None = None,
                ff_flags: int | None = None) -> dict:
        """coh, inc, tot, paper spectra per bin for the given (or own) shape."""
        kind = self.ff_kind if ff_kind is None else int(ff_kind)
        width = self.ff_width if ff_width is None else float(ff_width)
        flags = self.ff_flags if ff_flags is None else int(ff_flags)
        nb = self.n_bins
        out = {k: np.zeros(nb) for k in ("coh", "inc", "tot", "paper")}
        _load().oracle_readout(nb, _p(self.bin_omega), _p(self.bin_dir), _p(self.acc),
                               _p(self.comp), kind, flags, width, _p(out["coh"]), _p(out["inc"]),
                               _p(out["tot"]), _p(out["paper"]))
        return out


def accumulate_particles(bin_omega, bin_dir, r, beta, beta_dot, t, dt, a=None) -> np.ndarray:
    """Test-only per-particle integrals a_k = sum dt A_k e^{i phi_k}: [N][n_bins][3] complex."""
    bo, bdir = _f64(bin_omega).ravel(), _f64(bin_dir).reshape(-1, 3)
    r, beta, bd = _f64(r), _f64(beta), _f64(beta_dot)
    N = r.size // 3
    if a is None:
        a = np.zeros((N, bo.shape[0], 6))
    assert a.flags.c_contiguous and a.dtype == np.float64
    _load().oracle_accumulate_particles(bo.shape[0], _p(bo), _p(bdir), N, _p(r), _p(beta),
                                        _p(bd), float(t), float(dt), _p(a))
    return a


def complex_particles(a: np.ndarray) -> np.ndarray:
    return a[..., 0::2] + 1j * a[..., 1::2]


def species_spectra(accs, ffs) -> dict:
    """Spectra of a population made of several species (Sec. 3.2 applied per
    particle class): accs[s] holds species s's sums on a common bin list and
    ffs[s] = (kind, width[, flags]) its macro-particle shape.  The coherent
    amplitudes of all species add before the square; the incoherent part is a
    sum over species:
        coh = K0 |sum_s f_s U_s|^2,  inc = K0 sum_s (1 - f_s^2) |V_s|^2."""
    accs = list(accs)
    a0 = accs[0]
    nb = a0.n_bins
    u = np.zeros((nb, 3), dtype=complex)
    inc = np.zeros(nb)
    for acc, ff in zip(accs, ffs, strict=True):
        assert np.array_equal(acc.bin_omega, a0.bin_omega) and np.array_equal(acc.bin_dir, a0.bin_dir)
        kind, width = int(ff[0]), float(ff[1])
        flags = int(ff[2]) if len(ff) > 2 else 0
        f = np.array([form_factor_dir(kind, flags, width, om, n)
                      for om, n in zip(acc.bin_omega, acc.bin_dir)])
        amp = acc.amplitudes()
        u += f[:, None] * amp["U"]
        inc += (1.0 - f ** 2) * np.sum(np.abs(amp["V"]) ** 2, axis=1)
    coh = k0() * np.sum(np.abs(u) ** 2, axis=1)
    inc = k0() * inc
    return {"coh": coh, "inc": inc, "tot": coh + inc}
