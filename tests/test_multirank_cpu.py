"""World-size-2 gloo ranks on the CPU: particles sharded across ranks, per-rank
amplitudes merged on rank 0 in rank order, timing reduced with max.  The FP64
oracle stands in for each rank's engine (no GPU here); its amplitude arrays
play the role of the exported state blob."""
import os
import pickle
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1802_03972_gb300.multirank import shard_bounds


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


def _worker(rank, world, port, out_path):
    import torch.distributed as dist

    import oracle
    from paper_1802_03972_gb300 import inputs
    from paper_1802_03972_gb300.multirank import max_over_ranks, merge_to_root, shard_bounds
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
    state = acc.acc + acc.comp
    merged = [state.copy()]

    def merge(blob):
        merged[0] += pickle.loads(blob)

    n = merge_to_root(pickle.dumps(state), merge)
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
    want = full.acc + full.comp
    np.testing.assert_allclose(res["merged"], want, rtol=1e-11, atol=1e-11 * np.abs(want).max())
