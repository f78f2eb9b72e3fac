"""Wide calls: particles spread far beyond the fast phase range (|omega dtau|
up to 2^21 turns about one reference point: 40 um at 1e20 rad/s), as in the
in-situ use of Sec. 3.3 where one call holds all macro-particles of a domain.
The library sorts such a call's particles along the grid's mean direction,
writes their records relative to the first particle of each 256-particle
group and rotates each tile's sums by the group's reference phase, so the
tiles stay on the FP32 phase path.  Every case is checked against the FP64
oracle under both parity gates; results are deterministic and the same alone
and in a batch."""
import numpy as np
import pytest

import oracle
from gpu_util import assert_parity, to_dev
from paper_1802_03972_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1802_03972_gb300 import build as _build  # noqa: E402

_build.build()
from paper_1802_03972_gb300 import rad  # noqa: E402

C = 299792458.0


def wide_bunch(n, half_length, seed, n_omega=64, n_side=2, omega_hi=1e20):
    """n particles uniform over +-half_length along z (2 um transverse), gamma
    ~ 300 moving along z with small transverse velocities and accelerations."""
    rng = np.random.default_rng(seed)
    r = np.stack([rng.normal(0, 2e-6, n), rng.normal(0, 2e-6, n),
                  rng.uniform(-half_length, half_length, n)])
    b = np.stack([rng.normal(0, 1e-3, n), rng.normal(0, 1e-3, n), np.zeros(n)])
    b[2] = np.sqrt(1 - 1.1e-5 - b[0] ** 2 - b[1] ** 2)
    bd = rng.normal(0, 1e13, (3, n))
    w = rng.uniform(1e3, 1e5, n)
    omega = inputs.omega_log(1e16, omega_hi, n_omega)
    dirs = inputs.dirs_grid(0.01, n_side, n_side)
    return omega, dirs, r, b, bd, w


def steps(r, b, bd, w, n_steps=3, dt=1e-16):
    for s in range(n_steps):
        yield r + b * C * s * dt, b, bd, w, s * dt, dt


def run_pair(omega, dirs, data, ff=(oracle.FF_GAUSS, 0.1e-6), tile=None, flags=0):
    bo, bdir = oracle.grid_bins(omega, dirs)
    acc = oracle.Accumulator(bo, bdir, ff[0], ff[1])
    ctx = rad.Context(omega, dirs, ff[0], ff[1], ff_flags=flags)
    if tile is not None:
        ctx.set_tile(*tile)
    for r, b, bd, w, t, dt in data:
        acc.accumulate(r, b, bd, w, t, dt)
        ctx.accumulate(to_dev(r), to_dev(b), to_dev(bd), to_dev(w), t, dt)
    shape = (dirs.shape[0], omega.shape[0])
    return ctx, acc, shape


@pytest.mark.parametrize("variant", [0, 1, 2, 3, 4, 5, 7, 8, 9])
def test_two_millimetre_bunch_all_variants(variant):
    """20000 particles over 2 mm at omega up to 1e20 rad/s: about 50 times the
    fast range about one reference, a few microns per sorted group."""
    omega, dirs, r, b, bd, w = wide_bunch(20000, 1e-3, seed=31)
    ctx, acc, shape = run_pair(omega, dirs, list(steps(r, b, bd, w)), tile=(variant, 0, 0))
    ref = {k: v.reshape(shape) for k, v in acc.spectra().items()}
    got = dict(zip(("coh", "inc", "tot"), ctx.spectrum()))
    for k in ("tot", "coh", "inc"):
        assert_parity(got[k], ref[k], what=f"variant {variant} {k}")


def test_wide_call_is_deterministic_and_ragged():
    """A ragged particle count (not a multiple of the 256-particle group) and
    many directions per tile; two runs give the same bytes."""
    omega, dirs, r, b, bd, w = wide_bunch(7777, 5e-4, seed=32, n_omega=40, n_side=3)
    data = list(steps(r, b, bd, w))
    ctx, acc, shape = run_pair(omega, dirs, data)
    ref = {k: v.reshape(shape) for k, v in acc.spectra().items()}
    first = ctx.spectrum()
    for k, g in zip(("coh", "inc", "tot"), first):
        assert_parity(g, ref[k], what=k)
    again, _, _ = run_pair(omega, dirs, data)
    for x, y in zip(first, again.spectrum()):
        np.testing.assert_array_equal(x, y)


def test_wide_literal_sum():
    omega, dirs, r, b, bd, w = wide_bunch(6000, 1e-3, seed=33, n_omega=48)
    ctx, acc, shape = run_pair(omega, dirs, list(steps(r, b, bd, w)), flags=rad.FF_LITERAL)
    ref = acc.spectra()["paper"].reshape(shape)
    assert_parity(ctx.spectrum_literal(), ref, what="literal")


def test_wide_call_with_invalid_particles():
    """Invalid particles (NaN position, |beta| > 1) in a wide call: reported
    once, skipped, wherever the sort puts them."""
    omega, dirs, r, b, bd, w = wide_bunch(3000, 1e-3, seed=34)
    good = list(steps(r, b, bd, w, n_steps=2))
    bo, bdir = oracle.grid_bins(omega, dirs)
    acc = oracle.Accumulator(bo, bdir, oracle.FF_GAUSS, 0.1e-6)
    ctx = rad.Context(omega, dirs, rad.FF_GAUSS, 0.1e-6)
    for r_, b_, bd_, w_, t, dt in good:
        acc.accumulate(r_, b_, bd_, w_, t, dt)
        rb = np.concatenate([r_, [[np.nan, 0.0], [0.0, 0.0], [0.0, 5e-4]]], 1)
        bb = np.concatenate([b_, [[0.0, 0.0], [0.0, 0.0], [0.5, 1.5]]], 1)
        bdb = np.concatenate([bd_, np.ones((3, 2)) * 1e13], 1)
        wb = np.concatenate([w_, [10.0, 10.0]])
        ctx.accumulate(to_dev(rb), to_dev(bb), to_dev(bdb), to_dev(wb), t, dt)
    with pytest.raises(rad.RadError) as ei:
        ctx.spectrum()
    assert ei.value.status == rad.RAD_EDATA
    shape = (dirs.shape[0], omega.shape[0])
    ref = {k: v.reshape(shape) for k, v in acc.spectra().items()}
    for k, g in zip(("coh", "inc", "tot"), ctx.spectrum()):
        assert_parity(g, ref[k], what=k)


def test_wide_job_in_a_batch_equals_alone():
    """A wide job batched with two compact ones: every job's result is the same
    bytes as its standalone run, and the wide one matches the oracle."""
    omega, dirs, r, b, bd, w = wide_bunch(9000, 1e-3, seed=35)
    compact = [inputs.lwfa_bunch(n_particles=n, n_omega=64, n_side=2, seed=36 + n) for n in (700, 2500)]
    ctxs = [rad.Context(omega, dirs, rad.FF_GAUSS, 0.1e-6)] + [
        rad.Context(wl.omega, wl.dirs, wl.ff_kind, wl.ff_width) for wl in compact]
    alone = [rad.Context(omega, dirs, rad.FF_GAUSS, 0.1e-6)] + [
        rad.Context(wl.omega, wl.dirs, wl.ff_kind, wl.ff_width) for wl in compact]
    batch = rad.Batch(ctxs)
    wide_data = list(steps(r, b, bd, w))
    for s in range(3):
        r_, b_, bd_, w_, t, dt = wide_data[s]
        dev = [[to_dev(x) for x in (r_, b_, bd_, w_)]]
        times = [(t, dt)]
        for wl in compact:
            st = wl.step(s)
            dev.append([to_dev(x) for x in (st.r, st.beta, st.beta_dot, st.w)])
            times.append((st.t, st.dt))
        batch.accumulate([rad.make_step(d[3].shape[0], *d, *tt) for d, tt in zip(dev, times)])
        for c, d, tt in zip(alone, dev, times):
            c.accumulate(*d, *tt)
    batch.sync()
    for a, c in zip(alone, ctxs):
        for x, y in zip(a.spectrum(), c.spectrum()):
            np.testing.assert_array_equal(x, y)
    bo, bdir = oracle.grid_bins(omega, dirs)
    acc = oracle.Accumulator(bo, bdir, oracle.FF_GAUSS, 0.1e-6)
    for r_, b_, bd_, w_, t, dt in wide_data:
        acc.accumulate(r_, b_, bd_, w_, t, dt)
    shape = (dirs.shape[0], omega.shape[0])
    for k, g in zip(("coh", "inc", "tot"), ctxs[0].spectrum()):
        assert_parity(g, acc.spectra()[k].reshape(shape), what=k)
    batch.close()


def test_compact_and_wide_calls_alternate_on_one_context():
    """The wide flag belongs to the call: a context fed a compact call, a wide
    one, a compact one and a wide one (different particle counts) matches the
    oracle fed the same calls."""
    omega, dirs, r, b, bd, w = wide_bunch(5000, 1e-3, seed=37)
    compact = inputs.BetatronBunch(3000, seed=38)
    bo, bdir = oracle.grid_bins(omega, dirs)
    acc = oracle.Accumulator(bo, bdir, oracle.FF_GAUSS, 0.1e-6)
    ctx = rad.Context(omega, dirs, rad.FF_GAUSS, 0.1e-6)
    wide_data = list(steps(r, b, bd, w, n_steps=2))
    for s in range(4):
        if s % 2 == 0:
            st = compact.step(s * 1e-16, 1e-16)
            call = (st.r.reshape(3, -1), st.beta.reshape(3, -1), st.beta_dot.reshape(3, -1), st.w,
                    st.t, st.dt)
        else:
            call = wide_data[s // 2]
        acc.accumulate(*call)
        ctx.accumulate(*(to_dev(np.ascontiguousarray(x)) for x in call[:4]), call[4], call[5])
    shape = (dirs.shape[0], omega.shape[0])
    for k, g in zip(("coh", "inc", "tot"), ctx.spectrum()):
        assert_parity(g, acc.spectra()[k].reshape(shape), what=k)


def test_wide_bunch_through_the_in_situ_coupling():
    """rad_push_step with a wide bunch (beta_dot differenced on the device): the
    same spectra as feeding the differenced beta_dot to rad_accumulate."""
    omega, dirs, r, b, bd, w = wide_bunch(4000, 1e-3, seed=39)
    dt = 1e-16
    # beta rotating slowly so that the differences are not zero
    rots = [np.array([np.cos(1e-3 * s), np.sin(1e-3 * s)]) for s in range(4)]
    betas = []
    for c, s_ in rots:
        bb = b.copy()
        bb[0], bb[1] = c * b[0] - s_ * b[1], s_ * b[0] + c * b[1]
        betas.append(bb)
    rs = [r + betas[s] * C * s * dt for s in range(4)]
    push = rad.Context(omega, dirs, rad.FF_GAUSS, 0.1e-6)
    for s in range(4):
        push.push_step(to_dev(rs[s]), to_dev(betas[s]), to_dev(w), s * dt, dt)
    push.push_flush()
    ref = rad.Context(omega, dirs, rad.FF_GAUSS, 0.1e-6)
    for s in range(4):
        if s == 0:
            bdot = (betas[1] - betas[0]) / dt
        elif s == 3:
            bdot = (betas[3] - betas[2]) / dt
        else:
            bdot = (betas[s + 1] - betas[s - 1]) / (2 * dt)
        ref.accumulate(to_dev(rs[s]), to_dev(betas[s]), to_dev(bdot), to_dev(w), s * dt, dt)
    for a_, b_ in zip(push.spectrum(), ref.spectrum()):
        assert_parity(a_, b_, what="push vs accumulate")


def test_wide_bunch_over_fifty_steps():
    """A 2 mm bunch moving at ~c for 50 steps: every call is sorted afresh and
    read against its own reference point; the sum over time stays within both
    gates (read out after 10 and 50 steps)."""
    omega, dirs, r, b, bd, w = wide_bunch(5000, 1e-3, seed=40, n_omega=64, n_side=2)
    bo, bdir = oracle.grid_bins(omega, dirs)
    acc = oracle.Accumulator(bo, bdir, oracle.FF_GAUSS, 0.1e-6)
    ctx = rad.Context(omega, dirs, rad.FF_GAUSS, 0.1e-6)
    shape = (dirs.shape[0], omega.shape[0])
    for s, (r_, b_, bd_, w_, t, dt) in enumerate(steps(r, b, bd, w, n_steps=50)):
        acc.accumulate(r_, b_, bd_, w_, t, dt)
        ctx.accumulate(to_dev(r_), to_dev(b_), to_dev(bd_), to_dev(w_), t, dt)
        if s + 1 in (10, 50):
            for k, g in zip(("coh", "inc", "tot"), ctx.spectrum()):
                assert_parity(g, acc.spectra()[k].reshape(shape), what=f"{k} after {s + 1} steps")


@pytest.mark.parametrize("variant", [0, 8, 9])
def test_wide_call_tiles_on_the_fp64_path(variant):
    """A bunch 1 mm wide across the sort axis as well as along it, observed over
    +-0.3 rad: sorting along the mean direction cannot make the groups compact
    for the oblique directions, so some tiles take the per-update FP64 phase
    path with their group's reference time added, others the rotated FP32
    path; all against the oracle."""
    # 30000 particles: groups of 256 span ~8 um along z (fast for the directions
    # with no x component), ~1 mm across it (FP64 path for the oblique ones);
    # 512 frequencies make every tile one direction, so both paths occur
    rng = np.random.default_rng(41)
    n = 30000
    r = np.stack([rng.uniform(-5e-4, 5e-4, n), rng.normal(0, 2e-6, n), rng.uniform(-5e-4, 5e-4, n)])
    b = np.stack([rng.normal(0, 1e-3, n), rng.normal(0, 1e-3, n), np.zeros(n)])
    b[2] = np.sqrt(1 - 1.1e-5 - b[0] ** 2 - b[1] ** 2)
    bd = rng.normal(0, 1e13, (3, n))
    w = rng.uniform(1e3, 1e5, n)
    omega = inputs.omega_log(1e16, 1e20, 512)
    dirs = inputs.dirs_grid(0.3, 3, 3)
    ctx, acc, shape = run_pair(omega, dirs, list(steps(r, b, bd, w, n_steps=2)), tile=(variant, 0, 0))
    ref = {k: v.reshape(shape) for k, v in acc.spectra().items()}
    for k, g in zip(("coh", "inc", "tot"), ctx.spectrum()):
        assert_parity(g, ref[k], what=f"variant {variant} {k}")


@pytest.mark.parametrize("n_side, rows", [(8, [2, 31, 32, 63]), (12, [2, 106, 107, 138, 139, 143])])
def test_wide_call_with_fine_tail_tiles(n_side, rows):
    """A wide call whose last tiles are fine-chunked: 20480 particles over 2 mm on
    512 omega, 10 coarse chunks per tile, so on GB300 (304 resident blocks) 32
    tiles take 40 chunks of 512 sorted particles each, rotated group by group in
    the wide instantiation.  On 8 x 8 directions (64 tiles) that is the last 32;
    on 12 x 12 (144 tiles) the last 5 take a second level of 80 chunks of 256
    particles after them.  Directions on both sides of each boundary against the
    oracle over all frequencies, 2 steps."""
    omega, dirs, r, b, bd, w = wide_bunch(20480, 1e-3, seed=61, n_omega=512, n_side=n_side)
    ctx = rad.Context(omega, dirs, oracle.FF_GAUSS, 0.1e-6)
    assert ctx.get_tile()[0] == 9
    bins = [(d, o) for d in rows for o in range(omega.shape[0])]
    bo, bdir = oracle.grid_bins(omega, dirs, bins)
    acc = oracle.Accumulator(bo, bdir, oracle.FF_GAUSS, 0.1e-6)
    for rr, bb, bbd, ww, t, dt in steps(r, b, bd, w, n_steps=2):
        acc.accumulate(rr, bb, bbd, ww, t, dt)
        ctx.accumulate(to_dev(rr), to_dev(bb), to_dev(bbd), to_dev(ww), t, dt)
    got = dict(zip(("coh", "inc", "tot"), ctx.spectrum()))
    ref = {k: v.reshape(len(rows), omega.shape[0]) for k, v in acc.spectra().items()}
    for k in ("tot", "coh", "inc"):
        assert_parity(got[k][rows], ref[k], what=f"{k} rows {rows}")
