"""In-situ coupling (rad_push_step): steps without beta_dot, differenced on the
device, against the oracle fed the same finite differences and against the
analytic beta_dot of the trajectory."""
import numpy as np
import pytest

from gpu_util import assert_parity, gpu_run, row_error, spectra_grid, to_dev
import oracle
from paper_1802_03972_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1802_03972_gb300 import build as _build  # noqa: E402

_build.build()
from paper_1802_03972_gb300 import rad  # noqa: E402


def fd_beta_dot(steps):
    """Forward difference at the first step, central in the interior, backward at the last."""
    out = []
    m = len(steps)
    for j in range(m):
        a, b = (j, j + 1) if j == 0 else ((j - 1, j) if j == m - 1 else (j - 1, j + 1))
        out.append((steps[b].beta - steps[a].beta) / (steps[b].t - steps[a].t))
    return out


def test_push_matches_oracle_with_finite_differences():
    wl = inputs.lwfa_bunch(n_particles=700, n_omega=64, n_side=4, seed=71)
    steps = [wl.step(s) for s in range(12)]
    bdots = fd_beta_dot(steps)
    bo, bd = oracle.grid_bins(wl.omega, wl.dirs)
    acc = oracle.Accumulator(bo, bd, wl.ff_kind, wl.ff_width)
    for st, bdt in zip(steps, bdots):
        acc.accumulate(st.r, st.beta, bdt, st.w, st.t, st.dt)
    ref = spectra_grid(acc, wl)
    ctx = rad.Context(wl.omega, wl.dirs, wl.ff_kind, wl.ff_width)
    for st in steps:
        ctx.push_step(to_dev(st.r), to_dev(st.beta), to_dev(st.w), st.t, st.dt)
    ctx.push_flush()
    coh, inc, tot = ctx.spectrum()
    for k, g in (("tot", tot), ("coh", coh), ("inc", inc)):
        assert_parity(g, ref[k], what=k)


def test_push_agrees_with_analytic_beta_dot():
    """On the helix workload (step 1e-17 s, helix period 1e-12 s) second-order
    differences reproduce the analytic acceleration: spectra within 1e-4."""
    wl = inputs.tiny_helix(n_particles=32, n_steps=200, n_omega=64, n_dir=8)
    exact = gpu_run(wl, range(wl.n_steps)).spectrum()
    ctx = rad.Context(wl.omega, wl.dirs, wl.ff_kind, wl.ff_width)
    for s in range(wl.n_steps):
        st = wl.step(s)
        ctx.push_step(st.r, st.beta, st.w, st.t, st.dt)  # host arrays
    ctx.push_flush()
    got = ctx.spectrum()
    assert row_error(got[2], exact[2]) <= 1e-4


def test_push_rejects_changing_particle_count():
    wl = inputs.lwfa_bunch(n_particles=100, n_omega=32, n_side=1, seed=72)
    ctx = rad.Context(wl.omega, wl.dirs, wl.ff_kind, wl.ff_width)
    st = wl.step(0)
    ctx.push_step(st.r, st.beta, st.w, st.t, st.dt)
    short = inputs.lwfa_bunch(n_particles=99, n_omega=32, n_side=1, seed=72).step(1)
    with pytest.raises(rad.RadError) as ei:
        ctx.push_step(short.r, short.beta, short.w, short.t, short.dt)
    assert ei.value.status == rad.RAD_EINVAL
    ctx.push_flush()  # only one step held: nothing to difference, no error
