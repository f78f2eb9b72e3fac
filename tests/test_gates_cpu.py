"""The parity gates of the GPU tests, checked on the CPU: the per-bin gate must
catch a few wrong low-intensity bins that the per-direction 2-norm lets pass,
and accept errors of the size the error model allows."""
import numpy as np

from gpu_util import BIN_AMP, BIN_REL, TOL_TOTAL, bin_excess, row_error


def spectrum(rows=4, n=512, seed=0):
    """Rows falling from 1 to ~1e-8 of their peak, like a radiation spectrum
    past its coherent peak, with a ripple of deep minima."""
    rng = np.random.default_rng(seed)
    x = np.linspace(0.0, 18.0, n)
    out = np.exp(-x)[None, :] * (1.0 + 0.9 * np.cos(3.0 * x))[None, :] ** 2
    return out * rng.uniform(0.5, 2.0, (rows, 1))


def test_few_wrong_low_bins_pass_the_norm_but_fail_the_bin_gate():
    ref = spectrum()
    got = ref.copy()
    m = ref.max(axis=1)
    # three bins near 1e-4 of their direction's peak, each 2 % off
    for row in (0, 2, 3):
        j = int(np.argmin(np.abs(ref[row] / m[row] - 1e-4)))
        got[row, j] *= 1.02
    assert row_error(got, ref) <= TOL_TOTAL
    assert bin_excess(got, ref) > 1.0


def test_errors_the_model_allows_pass():
    ref = spectrum(seed=1)
    rng = np.random.default_rng(2)
    m = ref.max(axis=1, keepdims=True)
    # a relative error of half the relative allowance on every bin, plus an
    # amplitude error of half BIN_AMP of the peak amplitude with a random sign
    s = np.sqrt(ref)
    amp_err = 0.5 * BIN_AMP * np.sqrt(m) * rng.choice([-1.0, 1.0], ref.shape)
    got = (s + amp_err) ** 2 * (1.0 + 0.5 * BIN_REL)
    assert bin_excess(got, ref) <= 1.0
    assert row_error(got, ref) <= TOL_TOTAL


def test_relative_error_at_the_peak_is_bounded_by_the_relative_term():
    ref = spectrum(seed=3)
    j = ref.argmax(axis=1)
    got = ref.copy()
    got[np.arange(ref.shape[0]), j] *= 1.0 + 3.0 * BIN_REL
    assert bin_excess(got, ref) > 1.0


def test_exact_zeros_must_match():
    ref = np.zeros((2, 8))
    ref[0] = 1.0
    assert bin_excess(ref.copy(), ref) == 0.0
    got = ref.copy()
    got[1, 3] = 1e-300
    assert bin_excess(got, ref) == float("inf")
    got = ref.copy()
    got[0, 0] = np.nan
    assert bin_excess(got, ref) == float("inf")
