"""Helpers shared by the GPU tests: run a workload through the CUDA library
(C ABI via the binding) and through the FP64 oracle on the same inputs."""
from __future__ import annotations

import numpy as np

import oracle
from paper_1802_03972_gb300 import inputs

TOL_TOTAL = 1e-5   # relative spectral error of the mixed path vs the FP64 oracle
TOL_FP64 = 1e-9    # plain FP64 kernel vs the oracle (different summation order only)
# Per-bin gate (every bin of every direction, each part separately):
#   |I - I_ref| <= BIN_REL I_ref + 2 BIN_AMP sqrt(I_ref M) + BIN_AMP^2 M,
# M = the direction's largest I_ref.  It is the intensity error of an amplitude
# S' = S (1 + e_r) + e_a with |e_r| <= BIN_REL / 2 (rounding of the bin's own sum)
# and |e_a| <= BIN_AMP |S_max| (errors of single terms -- sin/cos, the TF32
# split, the FP32 phase -- on sums whose scale is set by the direction's
# largest amplitude).  Bins far below their direction's peak get a relative
# bound that grows like sqrt(M / I_ref), as amplitude errors of that size must;
# a spectral null (I_ref = 0 with M = 0) must be matched exactly.
BIN_REL, BIN_AMP = 1e-5, 2e-6
BIN_REL_FP64, BIN_AMP_FP64 = 1e-9, 1e-10


def row_error(got, ref) -> float:
    """max over directions of ||I(n,.) - I_ref(n,.)||_2 / ||I_ref(n,.)||_2 (rows with
    I_ref = 0 must be 0 too)."""
    got = np.asarray(got).reshape(ref.shape)
    err = 0.0
    for g, r in zip(got, ref):
        nr = np.linalg.norm(r)
        if nr == 0.0:
            assert np.all(g == 0.0) or np.linalg.norm(g) < 1e-300
            continue
        err = max(err, np.linalg.norm(g - r) / nr)
    return err


def bin_excess(got, ref, rel: float = BIN_REL, amp: float = BIN_AMP) -> float:
    """Largest ratio over all bins of |I - I_ref| to the per-bin allowance (see
    BIN_REL, BIN_AMP); the gate passes when it is <= 1.  Rows are directions."""
    ref = np.asarray(ref, dtype=np.float64)
    ref2 = ref.reshape(ref.shape[0], -1) if ref.ndim > 1 else ref.reshape(1, -1)
    got2 = np.asarray(got, dtype=np.float64).reshape(ref2.shape)
    m = np.abs(ref2).max(axis=1, keepdims=True)
    allowed = rel * np.abs(ref2) + 2.0 * amp * np.sqrt(np.abs(ref2) * m) + amp * amp * m
    diff = np.abs(got2 - ref2)
    if not np.all(np.isfinite(got2)):
        return float("inf")
    zero = allowed == 0.0
    if np.any(diff[zero] != 0.0):
        return float("inf")
    return float(np.max(np.where(zero, 0.0, diff / np.where(zero, 1.0, allowed)), initial=0.0))


def assert_parity(got, ref, tol: float = TOL_TOTAL, what: str = "", fp64: bool = False) -> dict:
    """The two parity gates: per-direction 2-norm error <= tol, and every bin
    within its per-bin allowance.  Returns both figures."""
    row = row_error(got, ref)
    ex = bin_excess(got, ref, *((BIN_REL_FP64, BIN_AMP_FP64) if fp64 else (BIN_REL, BIN_AMP)))
    assert row <= tol and ex <= 1.0, f"{what}: row error {row:.3e} (gate {tol:g}), bin excess {ex:.3f}"
    return {"row": row, "bin_excess": ex}


def assert_sampled_bins(got: dict, ref: dict, bins, what: str = "") -> float:
    """The per-bin gate on sampled bins: got[k] is a GPU spectrum [n_dir][n_omega]
    and ref[k][i] the oracle's value at bins[i] = (direction, frequency); the
    direction's largest intensity, which the allowance scales with, is taken
    from the GPU's row (within 1e-5 of the oracle's by the other gate).
    Returns the largest share of an allowance used."""
    worst = 0.0
    for k, g in got.items():
        g = np.asarray(g)
        for i, (d, o) in enumerate(bins):
            m = float(np.abs(g[d]).max())
            r = float(ref[k][i])
            allowed = BIN_REL * r + 2.0 * BIN_AMP * np.sqrt(r * m) + BIN_AMP ** 2 * m
            diff = abs(float(g[d, o]) - r)
            assert diff <= allowed, f"{what} {k} bin {(d, o)}: {g[d, o]!r} vs {r!r}"
            if allowed > 0:
                worst = max(worst, diff / allowed)
    return worst


def to_dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def gpu_run(wl: inputs.Workload, steps, prec=0, ff=None, tile=None, host=False, ctx=None):
    """Accumulate `steps` (iterable of step indices) of a workload on the GPU; returns
    the context (caller reads spectra)."""
    from paper_1802_03972_gb300 import rad
    if ctx is None:
        ff = (wl.ff_kind, wl.ff_width) if ff is None else ff
        ctx = rad.Context(wl.omega, wl.dirs, ff[0], ff[1], prec=prec)
        if tile is not None:
            ctx.set_tile(*tile)
    for s in steps:
        st = wl.step(s)
        if host:
            ctx.accumulate(st.r, st.beta, st.beta_dot, st.w, st.t, st.dt)
        else:
            ctx.accumulate(to_dev(st.r), to_dev(st.beta), to_dev(st.beta_dot), to_dev(st.w),
                           st.t, st.dt)
    return ctx


def oracle_run(wl: inputs.Workload, steps, bins=None):
    bo, bd = oracle.grid_bins(wl.omega, wl.dirs, bins)
    acc = oracle.Accumulator(bo, bd, wl.ff_kind, wl.ff_width)
    for s in steps:
        st = wl.step(s)
        acc.accumulate(st.r, st.beta, st.beta_dot, st.w, st.t, st.dt)
    return acc


def spectra_grid(acc: oracle.Accumulator, wl: inputs.Workload, ff=None) -> dict:
    sp = acc.spectra(*(ff or (None, None, None)))
    return {k: v.reshape(wl.dirs.shape[0], wl.omega.shape[0]) for k, v in sp.items()}
