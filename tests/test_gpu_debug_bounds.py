"""The debug build (librad_debug.so, compiled with RAD_DEBUG_BOUNDS) checks
every global-memory index that depends on the library's own sizing: the
particle-record capacity behind each TMA copy and each pre-pass write, the
partial-sum slots of each work item and tile, the tile counters; the sorted
positions of wide calls are checked in every build.  A failed check would
make the next synchronising call fail.  A cross-section of the parity tests
(every kernel variant, ragged and multi-direction tiles, particle counts that
change between calls, edge sizes, batches and the server, wide calls alone and
in a batch, the allocation-free entry, whose status is read after every call)
runs against it in a separate process."""
import os
import re
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_parity_cross_section_on_the_debug_build():
    from paper_1802_03972_gb300 import build
    lib = build.build(debug=True)
    env = dict(os.environ, RAD_LIBRARY=lib, RAD_LOG="1")
    sel = ("all_variants or wide_warp or two_pass or changing or edge_cases or tiny_helix_mixed or fine_tail "
           "or batch_equals_standalone or graph_replay or server_results_equal or static_entry "
           "or smaller_grid or invalid_direction or two_millimetre or deterministic_and_ragged "
           "or wide_job_in_a_batch")
    cmd = [sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider", "-k", sel,
           os.path.join(ROOT, "tests", "test_gpu_parity.py"),
           os.path.join(ROOT, "tests", "test_gpu_batch_server.py"),
           os.path.join(ROOT, "tests", "test_gpu_wide.py"),
           os.path.join(ROOT, "tests", "test_zz_no_alloc.py")]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, (r.stdout[-3000:], r.stderr[-3000:])
    m = re.search(r"(\d+) passed", r.stdout)
    assert m and int(m.group(1)) >= 30, r.stdout[-2000:]
    assert "index check" not in r.stderr
