"""In-situ scale: 1e7 macro-particles from the LWFA bunch generator streamed in
chunks of 1e6 into one time step, 1024 log frequencies x 32 x 32 directions
(1.05e13 amplitude updates), read out with CIC and TSC shapes of 0.1 um.

Checks: chunked streaming equals a different chunking (linearity of the sum),
32 sampled bins equal the FP64 oracle within the per-bin allowance of the
other parity tests (the direction's largest intensity, which the per-bin gate
scales with, taken from the GPU's row), and the mixed-precision kernel equals
the plain FP64 kernel on a reduced grid with all 1e7 particles."""
import numpy as np
import pytest

import oracle
from gpu_util import assert_parity, assert_sampled_bins, to_dev
from paper_1802_03972_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1802_03972_gb300 import build as _build  # noqa: E402

_build.build()
from paper_1802_03972_gb300 import rad  # noqa: E402

N_TOTAL, N_CHUNK = 10_000_000, 1_000_000


@pytest.fixture(scope="module")
def bunch():
    chunks = []
    for i in range(N_TOTAL // N_CHUNK):
        b = inputs.BetatronBunch(N_CHUNK, seed=300 + i)
        st = b.step(0.0, 1e-16)
        chunks.append(st)
    return chunks


def feed(ctx, chunks, split=1):
    for st in chunks:
        n = st.n
        r, b, bd = (st.r.reshape(3, n), st.beta.reshape(3, n), st.beta_dot.reshape(3, n))
        for part in np.array_split(np.arange(n), split):
            lo, hi = part[0], part[-1] + 1
            ctx.accumulate(to_dev(np.ascontiguousarray(r[:, lo:hi])), to_dev(np.ascontiguousarray(b[:, lo:hi])),
                           to_dev(np.ascontiguousarray(bd[:, lo:hi])), to_dev(st.w[lo:hi]), st.t, st.dt)


def test_insitu_scale_chunked_sampled_and_shapes(bunch):
    omega = inputs.omega_log(1e14, 1e20, 1024)
    dirs = inputs.dirs_grid(0.01, 32, 32)
    ctx = rad.Context(omega, dirs, rad.FF_CIC, 0.1e-6)
    feed(ctx, bunch)
    cic = ctx.spectrum()
    tsc = ctx.spectrum(ff=(rad.FF_TSC, 0.1e-6))
    # linearity: the same particles in 5e5-particle calls
    ctx3 = rad.Context(omega, dirs, rad.FF_CIC, 0.1e-6)
    feed(ctx3, bunch, split=2)
    for a, b in zip(cic, ctx3.spectrum()):
        assert_parity(b, a, what="chunking")
    # sampled bins against the oracle (all 1e7 particles)
    rng = np.random.default_rng(4)
    bins = [(int(rng.integers(0, 1024)), int(rng.integers(0, 1024))) for _ in range(32)]
    bo, bd = oracle.grid_bins(omega, dirs, bins)
    acc = oracle.Accumulator(bo, bd, oracle.FF_CIC, 0.1e-6)
    for st in bunch:
        acc.accumulate(st.r, st.beta, st.beta_dot, st.w, st.t, st.dt)
    for shape, got in ((oracle.FF_CIC, cic), (oracle.FF_TSC, tsc)):
        assert_sampled_bins(dict(zip(("coh", "inc", "tot"), got)), acc.spectra(shape, 0.1e-6), bins,
                            what=f"shape {shape}")


def test_insitu_scale_mixed_vs_plain_fp64(bunch):
    omega = inputs.omega_log(1e14, 1e20, 16)
    dirs = inputs.dirs_grid(0.01, 4, 4)
    mixed = rad.Context(omega, dirs, rad.FF_TSC, 0.1e-6)
    plain = rad.Context(omega, dirs, rad.FF_TSC, 0.1e-6, prec=rad.PREC_FP64)
    feed(mixed, bunch)
    feed(plain, bunch)
    for a, b in zip(mixed.spectrum(), plain.spectrum()):
        assert_parity(a, b, what="mixed vs plain FP64")
