"""Per-species readout (rad_spectrum_species) against the oracle's
species_spectra: a population made of several particle classes, each
accumulated in its own context and read out with its own macro-particle shape
(Sec. 3.2 per species).  The coherent amplitudes of all species add before the
square, so the test uses species that overlap in space (their cross terms are
large) and species whose accumulators have different reference particles."""
import numpy as np
import pytest

import oracle
from gpu_util import TOL_FP64, TOL_TOTAL, assert_parity, gpu_run, oracle_run, row_error, to_dev
from paper_1802_03972_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1802_03972_gb300 import build as _build  # noqa: E402

_build.build()
from paper_1802_03972_gb300 import rad  # noqa: E402

STEPS = range(6)


def species_workloads():
    """Three species on one grid (80 frequencies, 5 x 5 directions over +-0.3 rad
    so the 3-D box shape depends on the direction): two share one bunch's
    particles (electrons and a co-moving second class), one is another bunch."""
    out = []
    for seed, n in ((31, 900), (31, 900), (37, 1300)):
        wl = inputs.lwfa_bunch(n_particles=n, n_omega=80, n_side=5, seed=seed)
        wl.dirs = inputs.dirs_grid(0.3, 5, 5)
        out.append(wl)
    return out


FFS = [(oracle.FF_GAUSS, 0.1e-6), (oracle.FF_CIC, 0.25e-6, oracle.FF_3D), (oracle.FF_TSC, 0.15e-6)]


@pytest.fixture(scope="module")
def reference():
    wls = species_workloads()
    accs = [oracle_run(wl, STEPS) for wl in wls]
    shape = (wls[0].dirs.shape[0], wls[0].omega.shape[0])
    ref = {k: v.reshape(shape) for k, v in oracle.species_spectra(accs, FFS).items()}
    sep = sum(spec_tot(a, ff) for a, ff in zip(accs, FFS)).reshape(shape)
    return wls, ref, sep


def spec_tot(acc, ff):
    return acc.spectra(ff[0], ff[1], ff[2] if len(ff) > 2 else 0)["tot"]


@pytest.mark.parametrize("prec", [rad.PREC_MIXED, rad.PREC_FP64])
def test_three_species_match_oracle(reference, prec):
    wls, ref, sep = reference
    # the cross terms between species matter at the tolerance by a wide margin
    assert row_error(sep, ref["tot"]) > 1e3 * TOL_TOTAL
    ctxs = [gpu_run(wl, STEPS, prec=prec) for wl in wls]
    coh, inc, tot = rad.spectrum_species(ctxs, FFS)
    tol = TOL_TOTAL if prec == rad.PREC_MIXED else TOL_FP64
    for k, got in (("coh", coh), ("inc", inc), ("tot", tot)):
        assert_parity(got, ref[k], tol, what=k, fp64=prec != rad.PREC_MIXED)
    # device outputs give the same bytes as host outputs
    dev = tuple(torch.zeros(wls[0].dirs.shape[0], wls[0].omega.shape[0], dtype=torch.float64,
                            device="cuda") for _ in range(3))
    rad.spectrum_species(ctxs, FFS, out=dev)
    for h, d in zip((coh, inc, tot), dev):
        np.testing.assert_array_equal(h, d.cpu().numpy())


def test_one_species_equals_single_readout():
    wl = species_workloads()[2]
    ctx = gpu_run(wl, STEPS)
    for ff in FFS:
        flags = ff[2] if len(ff) > 2 else 0
        want = ctx.spectrum(ff=(ff[0], ff[1], flags))
        got = rad.spectrum_species([ctx], [ff])
        for g, w in zip(got, want):
            # f^2 |U|^2 against |f U|^2: equal up to rounding, except where the
            # Gaussian's f^2 leaves the normal range (values ~1e-310)
            np.testing.assert_allclose(g, w, rtol=1e-14, atol=1e-15 * np.abs(w).max())


def test_bad_species_arguments():
    wls = species_workloads()
    a = gpu_run(wls[0], range(1))
    b = gpu_run(wls[1], range(1))
    other_grid = inputs.lwfa_bunch(n_particles=100, n_omega=80, n_side=5, seed=3)  # +-10 mrad
    c = gpu_run(other_grid, range(1))
    d = gpu_run(wls[2], range(1), prec=rad.PREC_FP64)
    ff = FFS[0]
    cases = [([a, a], [ff, ff]),                       # a context repeated
             ([a, c], [ff, ff]),                       # same sizes, other directions
             ([a, d], [ff, ff]),                       # precisions differ
             ([a, b], [ff, (7, 0.1e-6)]),              # no such shape
             ([a, b], [ff, (oracle.FF_GAUSS, -1.0)]),  # negative width
             ([a] * 17, [ff] * 17)]                    # more than 16 species
    for ctxs, ffs in cases:
        with pytest.raises(rad.RadError) as ei:
            rad.spectrum_species(ctxs, ffs)
        assert ei.value.status == rad.RAD_EINVAL, (len(ctxs), ffs)
    # the refused calls leave the contexts usable
    coh, inc, tot = rad.spectrum_species([a, b], [ff, FFS[2]])
    assert np.all(np.isfinite(tot)) and np.all(tot > 0)


def test_species_with_invalid_particles_reports_once_and_keeps_spectra():
    """A species that saw invalid particles (NaN position, |beta| > 1): the
    species readout writes the spectra of the valid particles and returns
    RAD_EDATA once; the next readout is clean and identical."""
    wls = species_workloads()
    ref_accs = [oracle_run(wl, range(2)) for wl in wls[:2]]
    shape = (wls[0].dirs.shape[0], wls[0].omega.shape[0])
    ref = {k: v.reshape(shape) for k, v in oracle.species_spectra(ref_accs, FFS[:2]).items()}
    good = gpu_run(wls[0], range(2))
    bad = rad.Context(wls[1].omega, wls[1].dirs, wls[1].ff_kind, wls[1].ff_width)
    for s in range(2):
        st = wls[1].step(s)
        r = np.concatenate([st.r.reshape(3, -1), np.array([[np.nan], [0.0], [0.0]])], 1)
        b = np.concatenate([st.beta.reshape(3, -1), np.array([[0.0], [0.0], [1.5]])], 1)
        bd = np.concatenate([st.beta_dot.reshape(3, -1), np.ones((3, 1)) * 1e13], 1)
        w = np.concatenate([st.w, [10.0]])
        bad.accumulate(to_dev(r), to_dev(b), to_dev(bd), to_dev(w), st.t, st.dt)
    first = tuple(np.zeros(shape) for _ in range(3))
    with pytest.raises(rad.RadError) as ei:
        rad.spectrum_species([good, bad], FFS[:2], out=first)
    assert ei.value.status == rad.RAD_EDATA
    again = rad.spectrum_species([good, bad], FFS[:2])  # reported once: now clean
    for k, a, b2 in zip(("coh", "inc", "tot"), first, again):
        np.testing.assert_array_equal(a, b2)
        assert_parity(a, ref[k], what=k)
