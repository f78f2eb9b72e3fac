"""Helpers shared by the GPU tests: run a workload through the CUDA library
(C ABI via the binding) and through the FP64 oracle on the same inputs."""
from __future__ import annotations

import numpy as np

import oracle
from paper_1802_03972_gb300 import inputs

TOL_TOTAL = 1e-5   # relative spectral error of the mixed path vs the FP64 oracle
TOL_FP64 = 1e-9    # plain FP64 kernel vs the oracle (different summation order only)


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
