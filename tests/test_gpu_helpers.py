"""Pieces of the accumulate kernel's device arithmetic, run through the same
device functions by the self-test entry points, against FP64 host values:

* stage 1 (per particle and direction): the float-float retarded-time offset
  -n.(r_k - r_0)/c and the transverse amplitude e_i . A of
  A = n x ((n - beta) x beta_dot) / (1 - beta.n)^2 (Eq. 1), weighted by w dt and
  sqrt(w) dt, including particles at gamma = 1e4 where 1 - beta.n cancels;
* the phase omega tau: the fast path (float-float product reduced exactly to
  (-pi, pi] plus cross terms) for |omega tau / 2 pi| < 2^21 turns, and the FP64
  wide path beyond.
"""
import numpy as np
import pytest

from gpu_util import to_dev
from paper_1802_03972_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1802_03972_gb300 import build as _build  # noqa: E402

_build.build()
from paper_1802_03972_gb300 import rad  # noqa: E402

C = 299792458.0


def wrap(x):
    return np.angle(np.exp(1j * x))


def amplitude(n, beta, bdot):
    """Eq. 1 amplitude in FP64, one particle per column: [3][N] arrays."""
    nb = np.broadcast_to(n[:, None], beta.shape)
    u = nb - beta
    cross = np.cross(u.T, bdot.T).T
    num = np.cross(nb.T, cross.T).T
    den = 1.0 - (beta * nb).sum(0)
    return num / den ** 2


@pytest.mark.parametrize("gamma", [50.0, 1e4])
def test_stage1_offset_and_amplitude(gamma):
    rng = np.random.default_rng(41)
    n = 4000
    omega = inputs.omega_log(1e14, 1e20, 32)
    dirs = inputs.dirs_grid(0.02, 5, 5)
    ctx = rad.Context(omega, dirs, rad.FF_GAUSS, 0.1e-6)
    r = rng.normal(0.0, 2e-6, (3, n)) + np.array([[1e-3], [-2e-3], [0.5]])  # far from the origin
    speed = np.sqrt(1.0 - 1.0 / gamma ** 2)
    theta = rng.normal(0.0, 0.005, (2, n))
    beta = speed * np.vstack([np.sin(theta[0]), np.sin(theta[1]),
                              np.sqrt(1.0 - np.sin(theta[0]) ** 2 - np.sin(theta[1]) ** 2)])
    bdot = rng.normal(0.0, 1e12, (3, n))
    w = rng.uniform(1e3, 1e5, n)
    t, dt = 3e-12, 1e-16
    for d in (0, 12, 24):
        out, basis = ctx.selftest_stage1(*(to_dev(a.ravel()) for a in (r, beta, bdot)), to_dev(w), t, dt, d)
        nvec = dirs[d]
        tau = -(nvec[:, None] * (r - r[:, :1])).sum(0) / C
        got = out[:, 0].astype(np.float64) + out[:, 1].astype(np.float64)
        scale = np.abs(r - r[:, :1]).max() / C
        assert np.max(np.abs(got - tau)) <= 1e-12 * scale
        assert np.all(out[:, 6] == 1.0)  # within the fast phase path
        A = amplitude(nvec, beta, bdot)
        e = basis.astype(np.float64)
        a_ref = e @ A  # (2, n): e_i . A
        mag = np.sqrt((A ** 2).sum(0))
        for col, wt in ((2, w * dt), (4, np.sqrt(w) * dt)):
            for i in range(2):
                err = np.abs(out[:, col + i] - wt * a_ref[i]) / (wt * mag)
                assert err.max() <= 2e-5, (d, col, i, err.max())
        # n . A = 0: the two transverse components carry all of |A|
        carried = np.sqrt(out[:, 2].astype(np.float64) ** 2 + out[:, 3].astype(np.float64) ** 2) / (w * dt)
        assert np.max(np.abs(carried / mag - 1.0)) <= 2e-5


def test_phase_fast_and_wide_paths():
    rng = np.random.default_rng(42)
    omega = inputs.omega_log(1e14, 1e20, 48)
    ctx = rad.Context(omega, inputs.dirs_grid(0.01, 2, 2), rad.FF_POINT, 0.0)
    nu = omega / (2 * np.pi)
    lim = 2.0 ** 21 / nu.max()          # fast path range at the highest frequency
    tau = np.concatenate([rng.uniform(-lim, lim, 400), [0.0, lim * 0.999, -lim * 0.999, 1e-30],
                          rng.uniform(-1e4 * lim, 1e4 * lim, 100)])
    th = tau.astype(np.float32)
    tl = (tau - th.astype(np.float64)).astype(np.float32)
    fast, wide = ctx.selftest_phase(th, tl)
    tt = th.astype(np.float64) + tl.astype(np.float64)
    turns = nu[:, None] * tt[None, :]
    ref = 2 * np.pi * (turns - np.rint(turns))
    in_range = np.abs(turns) < 2.0 ** 21
    err_fast = np.abs(wrap(fast.astype(np.float64) - ref))[in_range]
    assert err_fast.max() <= 2e-6, err_fast.max()
    assert np.all(np.abs(fast[in_range]) <= np.pi + 0.8)  # reduced, plus bounded cross terms
    err_wide = np.abs(wrap(wide.astype(np.float64) - ref))
    assert err_wide.max() <= 2e-6, err_wide.max()
