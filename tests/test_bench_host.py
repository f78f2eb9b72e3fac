"""Host-side pieces of the benchmark, on the CPU: the one-job-at-a-time FIFO
latencies it reports beside the serving legs, and the lookup of the committed
DRAM-traffic capture."""
import importlib.util
import json
import math
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_fifo_latencies_by_hand(bench):
    # arrivals 0, 1, 1.5 s; work 2, 1, 4 units at 1 unit/s:
    # job 0 runs 0-2 (2 s), job 1 waits, runs 2-3 (2 s), job 2 runs 3-7 (5.5 s)
    r = bench.fifo_latencies([0.0, 1.0, 1.5], [2.0, 1.0, 4.0], 1.0)
    assert r["p50_s"] == pytest.approx(2.0, abs=0)
    assert r["p99_s"] == pytest.approx(2.0 + 0.98 * 3.5, rel=1e-12)
    # an idle gap: the server waits for the next arrival
    r = bench.fifo_latencies([0.0, 10.0], [1.0, 1.0], 1.0)
    assert r["p50_s"] == pytest.approx(1.0, abs=0) and r["p99_s"] == pytest.approx(1.0, abs=0)


def test_traffic_lookup_matches_only_the_captured_kernel_and_tile(bench, tmp_path, monkeypatch):
    sha = bench.kernel_hash()
    cap = {"captures": [{"kernel_sha": sha, "tile": [3, 256, 2048], "dram_bytes_per_launch": 4.0e8,
                         "updates_per_launch": 1.0e10}]}
    f = tmp_path / "traffic.json"
    f.write_text(json.dumps(cap))
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(f))
    assert bench.traffic_per_launch(2.0e10, [3, 256, 2048]) == pytest.approx(8.0e8, rel=1e-12)
    assert bench.traffic_per_launch(1.0e10, [7, 512, 1536]) is None
    cap["captures"][0]["kernel_sha"] = "0" * 16
    f.write_text(json.dumps(cap))
    assert bench.traffic_per_launch(1.0e10, [3, 256, 2048]) is None


def test_committed_traffic_capture_is_well_formed(bench):
    caps = json.load(open(bench.TRAFFIC_FILE))["captures"]
    assert caps
    for c in caps:
        assert len(c["kernel_sha"]) == 16 and len(c["tile"]) == 3
        assert c["dram_bytes_per_launch"] == pytest.approx(c["dram_bytes_read"] + c["dram_bytes_write"])
        assert "--clock-control none" in c["command"]


def test_error_stats_by_hand(bench):
    ref = [[1.0, 2.0, 1e-9, 0.0], [0.0, 0.0, 0.0, 0.0]]
    got = [[1.0 + 1e-6, 2.0, 5e-9, 0.0], [0.0, 0.0, 0.0, 0.0]]
    r = bench.error_stats(got, ref)
    # row 0: ||(1e-6, 0, 4e-9, 0)|| / ||(1, 2, 1e-9, 0)||; the all-zero row counts as exact
    assert r["row"] == pytest.approx(math.hypot(1e-6, 4e-9) / math.sqrt(5.0 + 1e-18), rel=1e-9)
    # bins kept: >= 1e-6 of the row maximum, so 1e-9 and 0 are left out
    assert r["bins"] == 2 and r["bin_max"] == pytest.approx(1e-6, rel=1e-9)
    assert bench.error_stats([[0.0, 1.0]], [[0.0, 0.0]])["row"] == math.inf
