"""rad_accumulate_static, the entry point for callers that cannot allocate
device memory (for example a plug-in inside a simulation's time-step loop where
cudaMalloc is forbidden), against the context-based rad_accumulate.

The file name sorts last, so a run that stops at the first failure has run
every other test before this one.  The test passes alone in a fresh process and
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


def test_static_entry_matches_context_two_calls_in_a_row():
    wl = inputs.lwfa_bunch(n_particles=3000, n_omega=96, n_side=4, seed=77)
    n_omega, n_dir = wl.omega.shape[0], wl.dirs.shape[0]
    n_bins = n_omega * n_dir
    omega_d = torch.from_numpy(wl.omega).cuda()
    dirs_d = torch.from_numpy(np.ascontiguousarray(wl.dirs)).cuda()
    state = torch.zeros(16 * n_bins, dtype=torch.float32, device="cuda")
    ctx = rad.Context(wl.omega, wl.dirs, wl.ff_kind, wl.ff_width)
    for s in range(2):
        st = wl.step(s)
        dev = [torch.from_numpy(a).cuda() for a in (st.r, st.beta, st.beta_dot, st.w)]
        rad.accumulate_static(omega_d, dirs_d, *dev, st.t, st.dt, state)
        ctx.accumulate(*dev, st.t, st.dt)
        torch.cuda.synchronize()
        blob = ctx.state_export()
        ref = np.frombuffer(blob[-16 * n_bins * 4:], dtype=np.float32)
        got = state.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert row_errors(amplitudes(got, n_bins), amplitudes(ref, n_bins), n_dir, n_omega) <= TOL
    ctx.close()


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
