"""Synthetic analogue of the paper's single macro-particle spectra (Sec. 4):
one macro-particle of w electrons on a betatron-like trajectory, read out with
the point shape (purely coherent, w^2 scaling), with a vanishing form factor
(purely incoherent, w scaling) and with a Gaussian shape whose width is the
mean electron spacing n_e^(-1/3) at n_e = 1e19 cm^-3.  The form-factor
spectrum follows w^2 below and w above the transition, where the coherent and
incoherent parts cross at f^2 = 1 / (w + 1) (Table 1, Eq. 12); the paper's
rough estimate of the transition, omega ~ c n_e^(1/3) / 2, is reported beside
it (Sec. 4 gives about 15 omega_0 estimated and 10 omega_0 simulated).

The same macro-particle runs through the FP64 oracle: every readout (the
Gaussian shape's coherent, incoherent and total parts, the point shape and the
vanishing form factor) is gated against it per direction and per bin, and the
crossing is located on the oracle's spectra as well as on the GPU's."""
import math

import numpy as np
import pytest

import oracle
from gpu_util import assert_parity
from paper_1802_03972_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1802_03972_gb300 import build as _build  # noqa: E402

_build.build()
from paper_1802_03972_gb300 import rad  # noqa: E402

C = 299792458.0


def test_coherent_incoherent_transition_of_one_macro_particle():
    n_e = 1e19 * 1e6                  # m^-3
    sigma = n_e ** (-1.0 / 3.0)       # mean electron spacing, 4.6 nm
    w = 1e4
    bunch = inputs.BetatronBunch(1, seed=81, w_lo=w, w_hi=w, n_e_cm3=1e19, gamma0=100.0)
    omega = inputs.omega_log(1e14, 1e19, 200)
    dirs = np.array([[0.0, 0.0, 1.0]])
    ctx = rad.Context(omega, dirs, rad.FF_GAUSS, sigma)
    bo, bd = oracle.grid_bins(omega, dirs)
    acc = oracle.Accumulator(bo, bd, oracle.FF_GAUSS, sigma)
    for s in range(400):
        st = bunch.step(s * 2e-16, 2e-16)
        ctx.accumulate(st.r, st.beta, st.beta_dot, st.w, st.t, st.dt)
        acc.accumulate(st.r, st.beta, st.beta_dot, st.w, st.t, st.dt)
    coh, inc, tot = (x[0] for x in ctx.spectrum())
    pure_coh = ctx.spectrum(ff=(rad.FF_POINT, 0.0))[2][0]            # w^2 |a|^2
    # a 1 m Gaussian has f^2 = exp(-(omega sigma / c)^2) = 0 at every omega >= 1e14 rad/s
    pure_inc = ctx.spectrum(ff=(rad.FF_GAUSS, 1.0))[2][0]             # f = 0: w |a|^2
    ref = acc.spectra()
    for k, got in (("coh", coh), ("inc", inc), ("tot", tot)):
        assert_parity(got[None, :], ref[k][None, :], what=k)
    ref_coh = acc.spectra(oracle.FF_POINT, 0.0)["tot"]
    ref_inc = acc.spectra(oracle.FF_GAUSS, 1.0)["tot"]
    assert_parity(pure_coh[None, :], ref_coh[None, :], what="point shape")
    assert_parity(pure_inc[None, :], ref_inc[None, :], what="vanishing form factor")
    np.testing.assert_allclose(pure_inc * w, pure_coh, rtol=1e-5)
    f2 = np.exp(-(omega * sigma / C) ** 2)
    # the form-factor spectrum is the f^2-weighted mix of the two scalings (Eq. 12)
    np.testing.assert_allclose(tot, f2 * pure_coh + (1 - f2) * pure_inc, rtol=1e-5)
    low, high = f2 > 1 - 1e-4, f2 < 1e-12
    assert low.any() and high.any()
    np.testing.assert_allclose(tot[low], pure_coh[low], rtol=2e-4)
    np.testing.assert_allclose(tot[high], pure_inc[high], rtol=1e-5)
    # coherent and incoherent parts cross where w^2 f^2 = w (1 - f^2), on the
    # GPU's spectra and on the oracle's
    omega_t = C / sigma * math.sqrt(math.log(w + 1.0))
    for c_, i_ in ((coh, inc), (ref["coh"], ref["inc"])):
        cross = np.argmax(c_ < i_)
        assert omega[cross - 1] <= omega_t <= omega[cross]
    omega0 = 2 * math.pi * C / 0.8e-6  # an 800 nm laser
    estimate = C * n_e ** (1.0 / 3.0) / 2
    print(f"transition {omega_t / omega0:.1f} omega_0 (w = {w:g}); "
          f"estimate c n_e^(1/3)/2 = {estimate / omega0:.1f} omega_0")
