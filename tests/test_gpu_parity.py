"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances: relative spectral error per direction (2-norm over frequencies)
<= 1e-5 for the mixed-precision path on the total spectrum and on its
coherent and incoherent parts, and every bin within the per-bin allowance of
gpu_util (relative 1e-5 plus an amplitude error of 2e-6 of the direction's
largest amplitude); 1e-9 (per bin: 1e-9 and 1e-10) for the plain FP64 kernel.
"""
import math

import numpy as np
import pytest

import oracle
from gpu_util import (TOL_FP64, TOL_TOTAL, assert_parity, gpu_run, oracle_run, spectra_grid,
                      to_dev)
from paper_1802_03972_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1802_03972_gb300 import build as _build  # noqa: E402

_build.build()
from paper_1802_03972_gb300 import rad  # noqa: E402


def check(ctx, ref, tol=TOL_TOTAL, parts=("tot", "coh", "inc"), ff=None):
    coh, inc, tot = ctx.spectrum(ff=ff)
    got = {"coh": coh, "inc": inc, "tot": tot}
    errs = {}
    for k in parts:
        errs[k] = assert_parity(got[k], ref[k], tol, what=k, fp64=tol == TOL_FP64)
    return errs


@pytest.fixture(scope="module")
def helix():
    wl = inputs.tiny_helix()
    return wl, spectra_grid(oracle_run(wl, range(wl.n_steps)), wl)


def test_tiny_helix_mixed_and_fp64(helix):
    """64 point particles on helices, 1000 steps, 128 x 16 bins (full grid)."""
    wl, ref = helix
    ctx = gpu_run(wl, range(wl.n_steps))
    check(ctx, ref, parts=("tot", "coh"))
    assert np.all(ctx.spectrum()[1] == 0.0)  # point shape: no incoherent part
    ctx64 = gpu_run(wl, range(wl.n_steps), prec=rad.PREC_FP64)
    check(ctx64, ref, tol=TOL_FP64, parts=("tot", "coh"))


def test_tiny_helix_host_buffers_match_device(helix):
    wl, _ = helix
    a = gpu_run(wl, range(50))
    b = gpu_run(wl, range(50), host=True)
    for x, y in zip(a.spectrum(), b.spectrum()):
        np.testing.assert_array_equal(x, y)


def small_lwfa(n=2000, n_omega=100, n_side=8, seed=21):
    wl = inputs.lwfa_bunch(n_particles=n, n_omega=n_omega, n_side=n_side, seed=seed)
    return wl


@pytest.mark.parametrize("variant", [0, 1, 2, 3, 4, 5, 7, 8, 9])
def test_lwfa_small_full_grid_all_variants(variant):
    """LWFA-shaped bunch with weights, Gaussian form factor, ragged particle count
    (2000 = 31 x 64 + 16) and ragged frequency tile (100 of 128), 20 steps."""
    wl = small_lwfa()
    ref = spectra_grid(oracle_run(wl, range(20)), wl)
    ctx = gpu_run(wl, range(20), tile=(variant, 0, 0))
    check(ctx, ref)


def test_two_pass_variant_full_width_tile():
    """Variant 7 sweeps each staged particle tile in two frequency passes: 300
    frequencies give one 512-wide tile whose second pass is ragged (44 of 256),
    over 9 directions and a ragged particle count."""
    wl = small_lwfa(n=1500, n_omega=300, n_side=3, seed=22)
    ref = spectra_grid(oracle_run(wl, range(6)), wl)
    ctx = gpu_run(wl, range(6), tile=(7, 512, 0))
    assert ctx.get_tile()[:2] == (7, 512)
    check(ctx, ref)


@pytest.mark.parametrize("variant", [8, 9])
def test_wide_warp_variant_full_width_tile(variant):
    """Variants 8 and 9 give each warp four 16-frequency blocks (64 frequencies):
    300 frequencies give one 512-wide tile whose last warps are ragged or empty,
    over 9 directions and a ragged particle count; and 48 frequencies in a
    64-wide tile of 8 directions, the last tile holding one."""
    for n_omega, n_side, wt in ((300, 3, 512), (48, 3, 64)):
        wl = small_lwfa(n=1500, n_omega=n_omega, n_side=n_side, seed=23)
        ref = spectra_grid(oracle_run(wl, range(6)), wl)
        ctx = gpu_run(wl, range(6), tile=(variant, wt, 0))
        assert ctx.get_tile()[:2] == (variant, wt)
        check(ctx, ref)


def test_lwfa_readout_with_other_shapes():
    """One accumulation read out with CIC, TSC, QSC and point shapes (the shape
    enters at readout only)."""
    wl = small_lwfa(n=700, n_omega=64, n_side=4)
    acc = oracle_run(wl, range(10))
    ctx = gpu_run(wl, range(10))
    for kind, width in ((oracle.FF_CIC, 0.1e-6), (oracle.FF_TSC, 0.2e-6), (oracle.FF_QSC, 0.05e-6),
                        (oracle.FF_POINT, 0.0)):
        ref = spectra_grid(acc, wl, (kind, width))
        check(ctx, ref, ff=(kind, width), parts=("tot", "coh") + (("inc",) if kind else ()))


def test_readout_3d_box_form_factor():
    """Axis-aligned 3-D box shapes (RAD_FF_3D): the form factor depends on the
    direction; oblique directions over a wide cone so the product differs."""
    wl = small_lwfa(n=400, n_omega=64, n_side=1)
    wl.dirs = inputs.dirs_grid(0.6, 3, 3)  # +-0.6 rad: strongly oblique directions
    acc = oracle_run(wl, range(4))
    ctx = gpu_run(wl, range(4))
    for kind, width in ((oracle.FF_CIC, 0.3e-6), (oracle.FF_TSC, 0.2e-6)):
        ref = spectra_grid(acc, wl, (kind, width, oracle.FF_3D))
        check(ctx, ref, ff=(kind, width, rad.FF_3D))


def test_lwfa_full_size_sampled_rows():
    """Full LWFA size (1e5 macro-particles, 512 log omega, 16 x 16 directions) in the
    benchmark's launch configuration (the tile rad_tune picks for this shape, as the
    benchmark uses it), 4 steps; the oracle computes 3 sampled directions over all
    512 frequencies (the gated per-direction error)."""
    wl = inputs.lwfa_bunch()
    steps = range(0, 4)
    ctx = rad.Context(wl.omega, wl.dirs, wl.ff_kind, wl.ff_width)
    ctx.tune(wl.n_particles)
    gpu_run(wl, steps, ctx=ctx)
    coh, inc, tot = ctx.spectrum()
    rows = [0, 137, 255]
    bins = [(d, o) for d in rows for o in range(512)]
    ref = {k: v.reshape(len(rows), 512) for k, v in oracle_run(wl, steps, bins).spectra().items()}
    for k, g in (("tot", tot), ("coh", coh), ("inc", inc)):
        assert_parity(g[rows], ref[k], what=k)


@pytest.mark.parametrize("n_omega, n_side, rows", [
    (512, 8, [5, 31, 32, 63]),
    (256, 12, [3, 79, 80, 81, 143]),
    (512, 12, [5, 106, 107, 138, 139, 143]),
    (256, 16, [3, 181, 182, 245, 246, 247, 255]),
])
def test_fine_tail_tiles(n_omega, n_side, rows):
    """The fine-chunked last tiles of a job.  20480 macro-particles in 2048-particle
    coarse chunks, 10 per tile, with one direction per tile at 512 frequencies and
    two at 256 (variant 9's default tile at that width); on GB300 (304 resident
    blocks) each job fills the GPU twice over.  Level 0 takes 32 tiles in 40
    chunks of 512 particles; level 1 (80 chunks of 256) follows only where its
    5 tiles keep both levels within half the job: not on 64 tiles (8 x 8
    directions) or 72 (12 x 12 at 256), but on 144 (12 x 12 at 512: coarse
    directions up to 106, level 0 107-138, level 1 139-143) and 128 (16 x 16 at
    256: coarse up to 181, level 0 182-245, level 1 246-255).  Directions on
    both sides of each boundary, both directions of a two-direction tile, and
    the last direction, against the oracle over all frequencies, 2 steps."""
    wl = inputs.lwfa_bunch(n_particles=20480, n_omega=n_omega, n_side=n_side, seed=29)
    steps = range(2)
    ctx = gpu_run(wl, steps)
    assert ctx.get_tile()[0] == 9
    coh, inc, tot = ctx.spectrum()
    bins = [(d, o) for d in rows for o in range(n_omega)]
    ref = {k: v.reshape(len(rows), n_omega) for k, v in oracle_run(wl, steps, bins).spectra().items()}
    for k, g in (("tot", tot), ("coh", coh), ("inc", inc)):
        assert_parity(g[rows], ref[k], what=f"{k} rows {rows}")


def test_lwfa_full_size_256_steps():
    """Accuracy over the workload's horizon: the full LWFA bunch for 256 of its
    2048 steps in the benchmark's launch configuration (the tuned tile), read out
    after 16, 64 and 256 steps.  This covers Eq. 13's sum over time in the
    precision the kernel uses (per-call partial sums rotated by the reference
    phase and added into compensated FP32 state).  The oracle computes 2
    directions x all 512 frequencies; both gates hold at every readout, and the
    error does not grow with the step count."""
    wl = inputs.lwfa_bunch()
    ctx = rad.Context(wl.omega, wl.dirs, wl.ff_kind, wl.ff_width)
    ctx.tune(wl.n_particles)
    rows = [5, 200]
    n_om = wl.omega.shape[0]
    acc = oracle_run(wl, [], [(d, o) for d in rows for o in range(n_om)])
    errs = {}
    for s in range(256):
        st = wl.step(s)
        ctx.accumulate(to_dev(st.r), to_dev(st.beta), to_dev(st.beta_dot), to_dev(st.w), st.t, st.dt)
        acc.accumulate(st.r, st.beta, st.beta_dot, st.w, st.t, st.dt)
        if s + 1 in (16, 64, 256):
            got = dict(zip(("coh", "inc", "tot"), ctx.spectrum()))
            ref = {k: v.reshape(len(rows), n_om) for k, v in acc.spectra().items()}
            errs[s + 1] = {k: assert_parity(got[k][rows], ref[k], what=f"{k} after {s + 1} steps")
                           for k in ("tot", "coh", "inc")}
    # no drift: the error after 256 steps stays within 2x of the error after 16
    assert errs[256]["tot"]["row"] <= 2.0 * errs[16]["tot"]["row"] + 1e-7, errs
    ctx.close()


def test_edge_cases_small_sizes():
    """n = 1, n_omega = 1, n_dir = 1, zero-particle calls."""
    for n, no, nd in ((1, 1, 1), (1, 3, 2), (65, 1, 5), (3, 130, 1)):
        wl = inputs.lwfa_bunch(n_particles=n, n_omega=no, n_side=1, seed=n + no)
        wl.dirs = inputs.dirs_grid(0.01, nd, 1) if nd > 1 else np.array([[0.0, 0.0, 1.0]])
        ref = spectra_grid(oracle_run(wl, range(5)), wl)
        ctx = gpu_run(wl, range(5))
        z = to_dev(np.zeros(0))
        ctx.accumulate(to_dev(np.zeros((3, 0))), to_dev(np.zeros((3, 0))), to_dev(np.zeros((3, 0))),
                       z, 1e-15, 1e-16)
        check(ctx, ref)


@pytest.mark.parametrize("variant", [3, 8, 9])
def test_changing_particle_counts_between_calls(variant):
    """One context fed calls of 3000, 700, 3000, 257 and 1 particles with a fixed
    chunk of 512: the number of chunks, and so of partial-sum slots each tile's
    last arrival adds up (and then drops from L2), changes from call to call;
    every call must use only the slots it wrote."""
    wl = small_lwfa(n=3000, n_omega=200, n_side=3, seed=24)
    bo, bd = oracle.grid_bins(wl.omega, wl.dirs)
    acc = oracle.Accumulator(bo, bd, wl.ff_kind, wl.ff_width)
    ctx = rad.Context(wl.omega, wl.dirs, wl.ff_kind, wl.ff_width)
    ctx.set_tile(variant, 0, 512)
    for s, n in enumerate((3000, 700, 3000, 257, 1)):
        st = wl.step(s)
        cut = [a.reshape(3, -1)[:, :n] for a in (st.r, st.beta, st.beta_dot)]
        acc.accumulate(*cut, st.w[:n], st.t, st.dt)
        ctx.accumulate(*(to_dev(np.ascontiguousarray(a).ravel()) for a in cut), to_dev(st.w[:n]),
                       st.t, st.dt)
    ref = spectra_grid(acc, wl)
    check(ctx, ref)


def test_invalid_particles_reported_and_skipped():
    wl = small_lwfa(n=300, n_omega=64, n_side=2)
    good = oracle_run(wl, range(3))
    ref = spectra_grid(good, wl)
    from paper_1802_03972_gb300 import rad as R
    ctx = R.Context(wl.omega, wl.dirs, wl.ff_kind, wl.ff_width)
    for s in range(3):
        st = wl.step(s)
        # append two bad particles: NaN position and |beta| > 1
        r = np.concatenate([st.r.reshape(3, -1), np.array([[np.nan, 0.0], [0.0, 0.0], [0.0, 0.0]])], 1)
        b = np.concatenate([st.beta.reshape(3, -1), np.array([[0.0, 0.0], [0.0, 0.0], [0.5, 1.5]])], 1)
        bd = np.concatenate([st.beta_dot.reshape(3, -1), np.ones((3, 2)) * 1e13], 1)
        w = np.concatenate([st.w, [10.0, 10.0]])
        ctx.accumulate(to_dev(r), to_dev(b), to_dev(bd), to_dev(w), st.t, st.dt)
    with pytest.raises(R.RadError) as ei:
        ctx.spectrum()
    assert ei.value.status == R.RAD_EDATA
    check(ctx, ref)  # reported once; the bad particles contributed nothing


def test_wide_bunch_uses_wide_phase_path():
    """Particles spread over 2 mm at omega up to 1e20 rad/s: |omega dtau| exceeds the
    fast path's 2^21 turns and the FP64 phase path must still match."""
    rng = np.random.default_rng(9)
    n = 200
    omega = inputs.omega_log(1e18, 1e20, 64)
    dirs = inputs.dirs_grid(0.01, 2, 2)
    r = np.stack([rng.normal(0, 1e-6, n), rng.normal(0, 1e-6, n), rng.uniform(-1e-3, 1e-3, n)])
    b = np.stack([rng.normal(0, 1e-3, n), rng.normal(0, 1e-3, n), np.zeros(n)])
    b[2] = np.sqrt(1 - 1e-5 - b[0] ** 2 - b[1] ** 2)
    bd = rng.normal(0, 1e13, (3, n))
    w = rng.uniform(1, 10, n)
    bo, bdir = oracle.grid_bins(omega, dirs)
    acc = oracle.Accumulator(bo, bdir)
    ctx = rad.Context(omega, dirs)
    for s in range(3):
        t = s * 1e-16
        acc.accumulate(r, b, bd, w, t, 1e-16)
        ctx.accumulate(to_dev(r), to_dev(b), to_dev(bd), to_dev(w), t, 1e-16)
        r = r + b * 299792458.0 * 1e-16
    ref = {k: v.reshape(4, 64) for k, v in acc.spectra().items()}
    check(ctx, ref, parts=("tot",))


def test_deterministic_bitwise():
    wl = small_lwfa(n=3000, n_omega=128, n_side=4)
    a = gpu_run(wl, range(4)).spectrum()
    b = gpu_run(wl, range(4)).spectrum()
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)


def test_large_time_offset():
    """A common time offset of 0.1 ns (omega t ~ 1e10 rad at 1e20 rad/s) only changes
    a common phase per call: the per-call reference keeps the fast path exact."""
    wl = small_lwfa(n=500, n_omega=64, n_side=2)
    shifted = inputs.Workload(wl.name, wl.omega, wl.dirs, wl.bunch, wl.n_steps, wl.dt, wl.ff_kind,
                              wl.ff_width)
    T = 1e-10

    def step(s, base=wl):
        st = base.step(s)
        st.t += T
        st.r = st.r.copy()
        st.r[2 * st.n:] += 299792458.0 * T  # bunch moved on by c T along z
        return st
    shifted.step = step
    ref = spectra_grid(oracle_run(shifted, range(4)), shifted)
    ctx = gpu_run(shifted, range(4))
    check(ctx, ref, parts=("tot",))


def test_profile_clock_reports_the_kernel_sm_clock():
    """rad_profile_clock: SM cycles over elapsed time of the profiled accumulate
    kernels, between 0.3 and 1.1 of the GPU's maximum clock; 0 after a read."""
    wl = small_lwfa(n=3000, n_omega=128, n_side=8)
    ctx = rad.Context(wl.omega, wl.dirs, wl.ff_kind, wl.ff_width)
    ctx.profile(True)
    gpu_run(wl, range(4), ctx=ctx)
    _, acc_ms, calls = ctx.profile_read()
    mhz = ctx.profile_clock()
    assert calls == 4 and acc_ms > 0
    assert 600.0 < mhz < 2300.0, mhz
    assert ctx.profile_clock() == 0.0


@pytest.mark.parametrize("variant", [8, 9])
def test_compact_call_at_the_edge_of_the_fast_range(variant):
    """A call whose particles reach 0.9 of the fast phase range from the reference
    point (the first particle) at the highest frequency: |omega dtau| up to
    0.9 x 2^21 turns at 1e20 rad/s, z from 0 to 35.5 um along the grid's axis.
    There the phase's float-float cross terms are largest (variant 9 forms them
    from TF32 splits on the tensor cores); the call is not wide, so every tile
    stays on the fast path.  Full grid (512 log omega up to 1e20 rad/s, 4 x 4
    directions) against the oracle, 2 steps."""
    rng = np.random.default_rng(71)
    n = 4000
    z = rng.uniform(0.0, 0.9 * 2 ** 21 / (1e20 / (2 * math.pi)) * 299792458.0, n)
    z[0] = 0.0
    r = np.stack([rng.normal(0, 2e-6, n), rng.normal(0, 2e-6, n), z])
    b = np.stack([rng.normal(0, 1e-3, n), rng.normal(0, 1e-3, n), np.zeros(n)])
    b[2] = np.sqrt(1 - 1.1e-5 - b[0] ** 2 - b[1] ** 2)
    bd = rng.normal(0, 1e13, (3, n))
    w = rng.uniform(1e3, 1e5, n)
    omega = inputs.omega_log(1e16, 1e20, 512)
    dirs = inputs.dirs_grid(0.01, 4, 4)
    bo, bdir = oracle.grid_bins(omega, dirs)
    acc = oracle.Accumulator(bo, bdir, oracle.FF_GAUSS, 0.1e-6)
    ctx = rad.Context(omega, dirs, oracle.FF_GAUSS, 0.1e-6)
    ctx.set_tile(variant, 0, 0)
    dt = 1e-16
    for s in range(2):
        rs = r + b * 299792458.0 * s * dt
        acc.accumulate(rs, b, bd, w, s * dt, dt)
        ctx.accumulate(to_dev(rs), to_dev(b), to_dev(bd), to_dev(w), s * dt, dt)
    got = dict(zip(("coh", "inc", "tot"), ctx.spectrum()))
    ref = {k: v.reshape(dirs.shape[0], omega.shape[0]) for k, v in acc.spectra().items()}
    for k in ("tot", "coh", "inc"):
        assert_parity(got[k], ref[k], what=f"variant {variant} {k}")
