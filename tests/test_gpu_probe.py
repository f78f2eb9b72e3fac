"""Pipe-throughput probes (rad_probe_peaks, rad_probe_tensor, rad_probe_loop): the rates they
report are per SM clock, so they must lie at or below the nominal per-SM widths
of the units (FP32 FMA 128 lanes, MUFU 16; legacy mma.sync TF32 about 500 multiply-adds) and
near them, and the effective clock must be a real SM clock."""
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1802_03972_gb300 import build as _build  # noqa: E402

_build.build()
from paper_1802_03972_gb300 import rad  # noqa: E402


def test_peaks_are_physical():
    p = rad.probe_peaks()
    ffma, ffma2, mufu, dfma = p[0], p[2], p[4], p[6]
    assert 64.0 <= ffma <= 128.0 * 1.02, ffma
    assert 64.0 <= ffma2 <= 128.0 * 1.02, ffma2
    assert 8.0 <= mufu <= 16.0 * 1.02, mufu
    assert 0.5 <= dfma <= 4.0, dfma
    for mhz in p[1:16:2]:
        assert 500.0 <= mhz <= 2200.0, mhz


def test_tensor_probe():
    q = rad.probe_tensor()
    assert 200.0 <= q[0] <= 560.0, q[0]   # mma.sync m16n8k8 TF32 MACs/clk/SM (~500 measured)
    tf32 = q[1:5]                                  # clocks per tcgen05.mma, N = 16, 64, 128, 256
    assert all(c > 0 for c in tf32)
    assert tf32[3] >= tf32[2] >= tf32[0] * 0.9     # wider N is never cheaper
    assert tf32[3] >= 128 * 256 * 8 / 2100.0       # at most ~2048 TF32 MACs per clock per SM
    assert all(c > 0 for c in q[5:7])
    assert 500.0 <= q[7] <= 2200.0, q[7]


def test_update_loop_probe():
    """The update loop's MUFU rate lies under the unit's 16 per SM clock in every
    mode, and taking work out of the loop (the split, the MMAs, both) never
    slows it: the decomposition behind the kernel's roofline fraction."""
    lp = rad.probe_loop()
    full8, no_split, no_mma, neither, full9 = lp[0], lp[2], lp[4], lp[6], lp[8]
    for rate in (full8, no_split, no_mma, neither, full9):
        assert 8.0 <= rate <= 16.0 * 1.02, lp
    assert neither >= max(no_split, no_mma) * 0.98, lp
    assert min(no_split, no_mma) >= full8 * 0.98, lp
    for mhz in lp[1:10:2]:
        assert 500.0 <= mhz <= 2200.0, mhz
