"""The paper's literal in-situ sum (Eq. 13 with the per-particle weight
F_k = sqrt(w + (w^2 - w) f^2) of Eq. 12) against the oracle's literal sum P."""
import numpy as np
import pytest

from gpu_util import assert_parity, oracle_run, row_error, spectra_grid, to_dev
import oracle
from paper_1802_03972_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1802_03972_gb300 import build as _build  # noqa: E402

_build.build()
from paper_1802_03972_gb300 import rad  # noqa: E402


def run_literal(wl, steps):
    ctx = rad.Context(wl.omega, wl.dirs, wl.ff_kind, wl.ff_width, ff_flags=rad.FF_LITERAL)
    for s in steps:
        st = wl.step(s)
        ctx.accumulate(to_dev(st.r), to_dev(st.beta), to_dev(st.beta_dot), to_dev(st.w), st.t, st.dt)
    return ctx


@pytest.mark.parametrize("kind,width", [(rad.FF_GAUSS, 0.1e-6), (rad.FF_TSC, 0.3e-6)])
def test_literal_sum_matches_oracle_with_unequal_weights(kind, width):
    """Weights uniform in [1e3, 1e5]: the literal spectrum matches the oracle's
    |P|^2 and the split outputs stay as before.  The two readings differ only by
    cross terms between particles of unequal weight in the bins where w f^2 is
    near 1 (per pair of heavy particles, the gap between the arithmetic and
    geometric mean of their weights), a few per mille there; the GPU must
    reproduce the oracle's difference in those bins."""
    wl = inputs.lwfa_bunch(n_particles=1500, n_omega=96, n_side=4, seed=61)
    wl.ff_kind, wl.ff_width = kind, width
    ref = spectra_grid(oracle_run(wl, range(6)), wl)
    ctx = run_literal(wl, range(6))
    lit = ctx.spectrum_literal()
    assert_parity(lit, ref["paper"], what="literal")
    coh, inc, tot = ctx.spectrum()
    assert_parity(tot, ref["tot"], what="tot")
    f2 = oracle.form_factor(kind, width, wl.omega) ** 2
    m = (f2 > 1e-6) & (f2 < 1e-2)
    assert m.sum() >= 3
    want = ref["paper"][:, m] - ref["tot"][:, m]
    assert row_error(ref["paper"][:, m], ref["tot"][:, m]) > 1e-3
    assert row_error(lit[:, m] - tot[:, m], want) <= 0.05


def test_literal_equals_split_for_equal_weights():
    wl = inputs.lwfa_bunch(n_particles=900, n_omega=64, n_side=4, seed=62)
    bunch = wl.bunch
    bunch.w = np.full(bunch.n, 4321.0)
    ctx = run_literal(wl, range(5))
    lit = ctx.spectrum_literal()
    tot = ctx.spectrum()[2]
    assert_parity(lit, tot, what="literal vs split")


def test_literal_checkpoint_and_restrictions():
    wl = inputs.lwfa_bunch(n_particles=500, n_omega=64, n_side=2, seed=63)
    a = run_literal(wl, range(3))
    blob = a.state_export()
    b = rad.Context(wl.omega, wl.dirs, wl.ff_kind, wl.ff_width, ff_flags=rad.FF_LITERAL)
    b.state_import(blob)
    np.testing.assert_array_equal(a.spectrum_literal(), b.spectrum_literal())
    plain = rad.Context(wl.omega, wl.dirs, wl.ff_kind, wl.ff_width)
    with pytest.raises(rad.RadError):
        plain.state_import(blob)          # payload shape differs
    with pytest.raises(rad.RadError):
        plain.spectrum_literal()          # not a literal context
    with pytest.raises(rad.RadError):
        rad.Batch([a])                    # literal contexts run on their own
    with pytest.raises(rad.RadError):
        rad.Context(wl.omega, wl.dirs, rad.FF_CIC, 0.1e-6, prec=rad.PREC_FP64, ff_flags=rad.FF_LITERAL)


def test_literal_merge_of_particle_shards():
    """Two contexts fed disjoint halves of the particles, merged (rad_state_merge),
    give the literal sum of one context fed all of them (amplitudes add before
    |.|^2; up to the order of floating-point sums)."""
    wl = inputs.lwfa_bunch(n_particles=1200, n_omega=64, n_side=4, seed=64)
    full = run_literal(wl, range(4))
    halves = []
    for lo, hi in ((0, 600), (600, 1200)):
        ctx = rad.Context(wl.omega, wl.dirs, wl.ff_kind, wl.ff_width, ff_flags=rad.FF_LITERAL)
        for s in range(4):
            st = wl.step(s)
            cut = [to_dev(a.reshape(3, -1)[:, lo:hi].ravel()) for a in (st.r, st.beta, st.beta_dot)]
            ctx.accumulate(*cut, to_dev(st.w[lo:hi]), st.t, st.dt)
        halves.append(ctx)
    halves[0].state_merge(halves[1].state_export())
    assert row_error(halves[0].spectrum_literal(), full.spectrum_literal()) <= 1e-6
    assert row_error(halves[0].spectrum()[2], full.spectrum()[2]) <= 1e-6
