"""rad_accumulate_static, the entry point for callers that cannot allocate
device memory (for example a plug-in inside a simulation's time-step loop where
cudaMalloc is forbidden), against the context-based rad_accumulate.

The file name sorts last, so a run that stops at the first failure has run
every other test before this one.  The tests pass alone in a fresh process and
after the other tests (the scratch array is shared by all calls and keeps the
previous call's contents)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1802_03972_gb300 import build as _build  # noqa: E402

_build.build()
from paper_1802_03972_gb300 import inputs, rad  # noqa: E402

TOL = 1e-5  # relative per-direction error, as in the other parity tests


def amplitudes(state_floats: np.ndarray, n_bins: int) -> np.ndarray:
    """[8][n_bins] compensated values sum - compensation of an accumulator array."""
    s = state_floats.reshape(16, n_bins).astype(np.float64)
    return s[:8] - s[8:]


def row_errors(a: np.ndarray, b: np.ndarray, n_dir: int, n_omega: int) -> float:
    """Max over directions of the relative 2-norm difference of |U|^2 and |V|^2."""
    err = 0.0
    for lo, hi in ((0, 4), (4, 8)):
        pa = (a[lo:hi] ** 2).sum(axis=0).reshape(n_dir, n_omega)
        pb = (b[lo:hi] ** 2).sum(axis=0).reshape(n_dir, n_omega)
        for ra, rb in zip(pa, pb):
            nb = np.linalg.norm(rb)
            if nb > 0:
                err = max(err, np.linalg.norm(ra - rb) / nb)
    return err


def device_inputs(wl, steps):
    """Grids and the steps' particle arrays, all on the device before any call."""
    om = torch.from_numpy(wl.omega).cuda()
    dirs = torch.from_numpy(np.ascontiguousarray(wl.dirs)).cuda()
    data = []
    for s in steps:
        st = wl.step(s)
        data.append(([torch.from_numpy(a).cuda() for a in (st.r, st.beta, st.beta_dot, st.w)],
                     st.t, st.dt))
    return om, dirs, data


def context_state(ctx, n_bins):
    blob = ctx.state_export()
    return np.frombuffer(blob[-16 * n_bins * 4:], dtype=np.float32)


def check_against_context(wl, steps, state, om, dirs, data):
    """Calls the static entry for each step and compares after each with a fresh
    context fed the same steps; the device status must be RAD_OK every time."""
    n_omega, n_dir = wl.omega.shape[0], wl.dirs.shape[0]
    n_bins = n_omega * n_dir
    ctx = rad.Context(wl.omega, wl.dirs, wl.ff_kind, wl.ff_width)
    for dev, t, dt in data:
        rad.accumulate_static(om, dirs, *dev, t, dt, state)
        assert rad.static_status() == rad.RAD_OK
        ctx.accumulate(*dev, t, dt)
        torch.cuda.synchronize()
        got = state.cpu().numpy()
        assert np.all(np.isfinite(got))
        ref = context_state(ctx, n_bins)
        assert row_errors(amplitudes(got, n_bins), amplitudes(ref, n_bins), n_dir, n_omega) <= TOL
    ctx.close()


def test_static_entry_matches_context_two_calls_in_a_row():
    wl = inputs.lwfa_bunch(n_particles=3000, n_omega=96, n_side=4, seed=77)
    n_bins = wl.omega.shape[0] * wl.dirs.shape[0]
    om, dirs, data = device_inputs(wl, range(2))
    state = torch.zeros(16 * n_bins, dtype=torch.float32, device="cuda")
    check_against_context(wl, range(2), state, om, dirs, data)


def test_static_entry_allocates_no_device_memory():
    """After a first call (which looks up the array's address), further calls
    leave the device's free memory unchanged."""
    wl = inputs.lwfa_bunch(n_particles=5000, n_omega=128, n_side=8, seed=78)
    n_bins = wl.omega.shape[0] * wl.dirs.shape[0]
    om, dirs, data = device_inputs(wl, range(4))
    state = torch.zeros(16 * n_bins, dtype=torch.float32, device="cuda")
    dev, t, dt = data[0]
    rad.accumulate_static(om, dirs, *dev, t, dt, state)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for dev, t, dt in data[1:]:
        rad.accumulate_static(om, dirs, *dev, t, dt, state)
        assert rad.static_status() == rad.RAD_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_smaller_grid_after_a_larger_one():
    """The shared array keeps the last call's tables and partial sums: a call on
    a smaller grid right after one on a larger grid must use only its own."""
    big = inputs.lwfa_bunch(n_particles=4000, n_omega=512, n_side=8, seed=79)
    small = inputs.lwfa_bunch(n_particles=1500, n_omega=40, n_side=3, seed=80)
    for wl in (big, small):
        n_bins = wl.omega.shape[0] * wl.dirs.shape[0]
        om, dirs, data = device_inputs(wl, range(2))
        state = torch.zeros(16 * n_bins, dtype=torch.float32, device="cuda")
        check_against_context(wl, range(2), state, om, dirs, data)


def test_invalid_direction_skips_the_step_and_is_reported():
    wl = inputs.lwfa_bunch(n_particles=2000, n_omega=64, n_side=2, seed=81)
    n_bins = wl.omega.shape[0] * wl.dirs.shape[0]
    om, dirs, data = device_inputs(wl, range(2))
    state = torch.zeros(16 * n_bins, dtype=torch.float32, device="cuda")
    dev, t, dt = data[0]
    rad.accumulate_static(om, dirs, *dev, t, dt, state)
    assert rad.static_status() == rad.RAD_OK
    before = state.cpu().numpy().copy()
    bad_dirs = dirs.clone()
    bad_dirs[1] = 0.0
    dev, t, dt = data[1]
    rad.accumulate_static(om, bad_dirs, *dev, t, dt, state)
    assert rad.static_status() == rad.RAD_EINVAL
    # every particle weighed zero: the compensated values are unchanged (adding
    # zero may only move rounding between a sum and its compensation)
    a0, a1 = amplitudes(before, n_bins), amplitudes(state.cpu().numpy(), n_bins)
    np.testing.assert_allclose(a1, a0, rtol=1e-6, atol=1e-7 * np.abs(a0).max())
    bad_om = om.clone()
    bad_om[3] = float("nan")
    rad.accumulate_static(bad_om, dirs, *dev, t, dt, state)
    assert rad.static_status() == rad.RAD_EINVAL
    assert np.all(np.isfinite(state.cpu().numpy()))
    # a valid call afterwards is reported OK again
    rad.accumulate_static(om, dirs, *dev, t, dt, state)
    assert rad.static_status() == rad.RAD_OK


def test_static_entry_rejects_sizes_beyond_its_limits():
    omega_d = torch.ones(8, dtype=torch.float64, device="cuda") * 1e15
    dirs_d = torch.tensor([[0.0, 0.0, 1.0]], dtype=torch.float64, device="cuda")
    state = torch.zeros(16 * 8, dtype=torch.float32, device="cuda")
    n = rad.STATIC_MAX_PARTICLES + 1
    big = torch.zeros(3 * n, dtype=torch.float64, device="cuda")
    w = torch.ones(n, dtype=torch.float64, device="cuda")
    with pytest.raises(rad.RadError) as ei:
        rad.accumulate_static(omega_d, dirs_d, big, big, big, w, 0.0, 1e-16, state)
    assert ei.value.status == rad.RAD_EINVAL
    many = torch.ones(rad.STATIC_MAX_OMEGA + 1, dtype=torch.float64, device="cuda")
    with pytest.raises(rad.RadError):
        rad.accumulate_static(many, dirs_d, big[:3], big[:3], big[:3], w[:1], 0.0, 1e-16, state)
