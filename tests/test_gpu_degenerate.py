"""Degenerate cases of the radiation sum on the GPU, checked against what the
mathematics fixes at any size (Eq. 1, Eq. 2, Eq. 12), on the FP32 and three
tensor-core kernel variants:

* beta_dot = 0: the amplitude n x ((n - beta) x beta_dot) / (1 - beta.n)^2
  vanishes, so every spectrum is exactly zero;
* N co-located, co-moving point particles of weight 1: the amplitudes add in
  phase, so the spectrum is N^2 times that of one;
* one macro-particle of weight w: the point shape (f = 1) gives w^2 times the
  weight-1 spectrum, a vanishing form factor (f = 0) gives w times it."""
import numpy as np
import pytest

from gpu_util import row_error, to_dev
from paper_1802_03972_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1802_03972_gb300 import build as _build  # noqa: E402

_build.build()
from paper_1802_03972_gb300 import rad  # noqa: E402

VARIANTS = [0, 3, 7, 8, 9]


def run(omega, dirs, steps, variant, ff=(rad.FF_POINT, 0.0), scale_w=1.0, repeat=1):
    """Accumulate the steps; each particle repeated `repeat` times in place and its
    weight multiplied by scale_w."""
    ctx = rad.Context(omega, dirs, ff[0], ff[1])
    ctx.set_tile(variant, 0, 0)
    for st in steps:
        cols = [np.repeat(a.reshape(3, -1), repeat, axis=1).ravel() for a in (st.r, st.beta, st.beta_dot)]
        w = np.repeat(st.w, repeat) * scale_w
        ctx.accumulate(*(to_dev(a) for a in cols), to_dev(w), st.t, st.dt)
    return ctx


def workload(n=7, seed=31):
    wl = inputs.lwfa_bunch(n_particles=n, n_omega=96, n_side=4, seed=seed)
    wl.bunch.w = np.ones(wl.bunch.n)
    return wl, [wl.step(s) for s in range(6)]


@pytest.mark.parametrize("variant", VARIANTS)
def test_zero_acceleration_gives_exactly_zero(variant):
    wl, steps = workload()
    for st in steps:
        st.beta_dot[:] = 0.0
    ctx = run(wl.omega, wl.dirs, steps, variant, ff=(rad.FF_GAUSS, 0.1e-6))
    for part in ctx.spectrum():
        assert np.all(part == 0.0)


@pytest.mark.parametrize("variant", VARIANTS)
def test_colocated_particles_add_coherently(variant):
    wl, steps = workload(n=1, seed=32)
    one = run(wl.omega, wl.dirs, steps, variant).spectrum()[2]
    for n in (2, 37):
        many = run(wl.omega, wl.dirs, steps, variant, repeat=n).spectrum()[2]
        assert row_error(many, n * n * one) <= 1e-5, n


@pytest.mark.parametrize("variant", VARIANTS)
def test_macro_particle_weight_scaling(variant):
    wl, steps = workload(n=1, seed=33)
    w = 5000.0
    base = run(wl.omega, wl.dirs, steps, variant).spectrum()[2]
    heavy = run(wl.omega, wl.dirs, steps, variant, scale_w=w)
    coh, inc, tot = heavy.spectrum()
    assert row_error(tot, w * w * base) <= 1e-5
    assert np.all(inc == 0.0)  # point shape: f = 1
    # a 1 m Gaussian has f = 0 at every frequency of the grid (>= 1e14 rad/s)
    coh0, inc0, tot0 = heavy.spectrum(ff=(rad.FF_GAUSS, 1.0))
    assert np.all(coh0 == 0.0)
    assert row_error(tot0, w * base) <= 1e-5
