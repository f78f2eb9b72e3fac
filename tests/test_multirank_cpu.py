"""World-size-2 gloo ranks on the CPU: particles sharded across ranks, per-rank
amplitudes sent to rank 0 as state blobs in the library's versioned format
(the format rad_state_export writes) and merged there in rank order by the
host-side merge, timing reduced with max.  The FP64 oracle stands in for each
rank's engine (no GPU here): its amplitudes fill an FP64 blob, which has the
same layout as an FP64 context's accumulators."""
import os
import pickle
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1802_03972_gb300.multirank import (make_state_blob, merge_state_blobs,
                                               parse_state_blob, shard_bounds)


def test_shard_bounds_partition():
    for n in (0, 1, 7, 100, 1001):
        for world in (1, 2, 3, 8):
            spans = [shard_bounds(n, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))
            sizes = [hi - lo for lo, hi in spans]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard_bounds(5, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def fp64_payload(acc):
    """[12][n_bins] FP64 payload of an oracle accumulator: U x, y, z then V x, y, z,
    each (re, im) -- the order of an FP64 context's accumulators."""
    return np.ascontiguousarray((acc.acc + acc.comp)[:, :12].T)


def _worker(rank, world, port, out_path):
    import torch.distributed as dist

    import oracle
    from paper_1802_03972_gb300 import inputs
    from paper_1802_03972_gb300.multirank import (make_state_blob, max_over_ranks,
                                                   merge_state_blobs, merge_to_root, shard_bounds)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    wl = inputs.lwfa_bunch(n_particles=301, n_omega=24, n_side=2, seed=17)
    bo, bd = oracle.grid_bins(wl.omega, wl.dirs)
    acc = oracle.Accumulator(bo, bd, wl.ff_kind, wl.ff_width)
    lo, hi = shard_bounds(wl.n_particles, rank, world)
    for s in range(4):
        st = wl.step(s)
        sl = slice(lo, hi)
        acc.accumulate(st.r.reshape(3, -1)[:, sl], st.beta.reshape(3, -1)[:, sl],
                       st.beta_dot.reshape(3, -1)[:, sl], st.w[sl], st.t, st.dt)
    blob = make_state_blob({"prec": 1, "n_omega": 24, "n_dir": 4, "elem_size": 8},
                           fp64_payload(acc))
    merged = [blob]

    def merge(other):
        merged[0] = merge_state_blobs(merged[0], other)

    n = merge_to_root(blob, merge)
    slowest = max_over_ranks(float(rank + 1))
    if rank == 0:
        with open(out_path, "wb") as f:
            pickle.dump({"merged": merged[0], "n": n, "slowest": slowest}, f)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_merge_equals_single_process(tmp_path):
    out = str(tmp_path / "rank0.pkl")
    mp.spawn(_worker, args=(2, _free_port(), out), nprocs=2, join=True)
    res = pickle.load(open(out, "rb"))
    assert res["n"] == 1 and res["slowest"] == 2.0

    import oracle
    from paper_1802_03972_gb300 import inputs
    wl = inputs.lwfa_bunch(n_particles=301, n_omega=24, n_side=2, seed=17)
    bo, bd = oracle.grid_bins(wl.omega, wl.dirs)
    full = oracle.Accumulator(bo, bd, wl.ff_kind, wl.ff_width)
    for s in range(4):
        st = wl.step(s)
        full.accumulate(st.r, st.beta, st.beta_dot, st.w, st.t, st.dt)
    head, got = parse_state_blob(res["merged"])
    assert head == {"prec": 1, "n_omega": 24, "n_dir": 4, "n_comp": 12, "elem_size": 8}
    want = fp64_payload(full)
    np.testing.assert_allclose(got, want, rtol=1e-11, atol=1e-11 * np.abs(want).max())


def test_mixed_blob_merge_adds_compensated_values():
    """Mixed blobs hold float32 (sum, compensation) pairs; merging adds each
    value sum - compensation with compensation, over many blobs as on many ranks."""
    rng = np.random.default_rng(5)
    head = {"prec": 0, "n_omega": 7, "n_dir": 3, "elem_size": 4}
    total = np.zeros((8, 21))
    blobs = []
    for _ in range(16):
        s = rng.normal(0.0, 1.0, (8, 21)).astype(np.float32)
        c = (rng.normal(0.0, 1.0, (8, 21)) * 1e-8).astype(np.float32)
        total += s.astype(np.float64) - c.astype(np.float64)
        blobs.append(make_state_blob(head, np.concatenate([s, c])))
    merged = blobs[0]
    for b in blobs[1:]:
        merged = merge_state_blobs(merged, b)
    h, arr = parse_state_blob(merged)
    assert h["n_comp"] == 16
    value = arr[:8].astype(np.float64) - arr[8:].astype(np.float64)
    np.testing.assert_allclose(value, total, rtol=0, atol=4 * np.finfo(np.float32).eps * 16)


def test_blob_header_checks():
    head = {"prec": 0, "n_omega": 2, "n_dir": 2, "elem_size": 4}
    blob = make_state_blob(head, np.zeros((16, 4), np.float32))
    assert len(blob) == 40 + 16 * 4 * 4
    with pytest.raises(ValueError):
        parse_state_blob(blob[:-4])
    with pytest.raises(ValueError):
        parse_state_blob(b"XXXX" + blob[4:])
    other = make_state_blob(dict(head, n_omega=4, n_dir=1), np.zeros((16, 4), np.float32))
    with pytest.raises(ValueError):
        merge_state_blobs(blob, other)
