"""One job's particles split across two processes (ranks of a gloo group, both
on cuda:0): each rank accumulates its shard_bounds slice of every step in its
own context; rank 0 merges rank 1's state with the library's real blobs
(rad_state_export, sent over the process group, rad_state_merge), the one
exchange of the particle partition at readout (amplitudes add before |.|^2,
Eq. 2).  The merged spectra must match the FP64 oracle under both parity gates
and the single-context run, and the host-side blob merge must give the
device merge's bytes.  The two processes' kernels never wait on each other:
the exchange is on the host, between steps."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from gpu_util import assert_parity, gpu_run, oracle_run, spectra_grid
from paper_1802_03972_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1802_03972_gb300 import build as _build  # noqa: E402

_build.build()

STEPS = range(5)


def workload():
    return inputs.lwfa_bunch(n_particles=3001, n_omega=96, n_side=4, seed=19)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out_dir):
    import torch
    import torch.distributed as dist

    from paper_1802_03972_gb300 import rad
    from paper_1802_03972_gb300.multirank import merge_to_root, shard_bounds
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    wl = workload()
    ctx = rad.Context(wl.omega, wl.dirs, wl.ff_kind, wl.ff_width)
    lo, hi = shard_bounds(wl.n_particles, rank, world)
    for s in STEPS:
        st = wl.step(s)
        part = [np.ascontiguousarray(a.reshape(3, -1)[:, lo:hi]) for a in (st.r, st.beta, st.beta_dot)]
        ctx.accumulate(*(torch.from_numpy(a).cuda() for a in part),
                       torch.from_numpy(st.w[lo:hi].copy()).cuda(), st.t, st.dt)
    own = ctx.state_export()
    np.save(os.path.join(out_dir, f"blob{rank}.npy"), np.frombuffer(own, dtype=np.uint8))
    merged = merge_to_root(own, ctx.state_merge)
    if rank == 0:
        coh, inc, tot = ctx.spectrum()
        np.savez(os.path.join(out_dir, "rank0.npz"), coh=coh, inc=inc, tot=tot,
                 merged=np.array([merged]),
                 state=np.frombuffer(ctx.state_export(), dtype=np.uint8))
    ctx.close()
    dist.barrier()
    dist.destroy_process_group()


def test_two_processes_merge_real_blobs(tmp_path):
    mp.spawn(_rank, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    res = np.load(tmp_path / "rank0.npz")
    assert int(res["merged"][0]) == 1
    wl = workload()
    ref = spectra_grid(oracle_run(wl, STEPS), wl)
    whole = gpu_run(wl, STEPS).spectrum()
    for k, i in (("coh", 0), ("inc", 1), ("tot", 2)):
        assert_parity(res[k], ref[k], what=f"merged {k} vs oracle")
        assert_parity(res[k], whole[i], what=f"merged {k} vs one context")
    # the host-side merge of the two ranks' blobs gives the device merge's bytes
    from paper_1802_03972_gb300.multirank import merge_state_blobs, parse_state_blob
    b0 = np.load(tmp_path / "blob0.npy").tobytes()
    b1 = np.load(tmp_path / "blob1.npy").tobytes()
    head, _ = parse_state_blob(b0)
    assert head == {"prec": 0, "n_omega": 96, "n_dir": 16, "n_comp": 16, "elem_size": 4}
    assert merge_state_blobs(b0, b1) == res["state"].tobytes()
