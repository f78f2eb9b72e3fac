"""Batched launches, CUDA-graph replay, checkpoint/merge, autotuning and the
continuous-batching server, all checked against standalone runs and the oracle."""
import time

import numpy as np
import pytest

from gpu_util import assert_parity, assert_sampled_bins, gpu_run, oracle_run, spectra_grid, to_dev
from paper_1802_03972_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1802_03972_gb300 import build as _build  # noqa: E402

_build.build()
from paper_1802_03972_gb300 import rad  # noqa: E402


def small_jobs():
    specs = [inputs.JobSpec(7000 + j, n, no, ns, 6, 100.0, 300.0, 2e-6)
             for j, (n, no, ns) in enumerate([(1500, 64, 4), (300, 256, 2), (4100, 128, 8), (64, 512, 1)])]
    return [s.workload() for s in specs]


def dev_steps(wl, s):
    st = wl.step(s)
    arrs = [to_dev(st.r), to_dev(st.beta), to_dev(st.beta_dot), to_dev(st.w)]
    return st, arrs


def test_batch_equals_standalone_bitwise_and_oracle():
    wls = small_jobs()
    alone = [gpu_run(wl, range(6)) for wl in wls]
    ctxs = [rad.Context(wl.omega, wl.dirs, wl.ff_kind, wl.ff_width) for wl in wls]
    batch = rad.Batch(ctxs)
    keep = []
    for s in range(6):
        steps = []
        for wl in wls:
            st, arrs = dev_steps(wl, s)
            keep.append(arrs)
            steps.append(rad.make_step(st.n, *arrs, st.t, st.dt))
        batch.accumulate(steps)
    batch.sync()
    for wl, a, c in zip(wls, alone, ctxs):
        for x, y in zip(a.spectrum(), c.spectrum()):
            np.testing.assert_array_equal(x, y)
        ref = spectra_grid(oracle_run(wl, range(6)), wl)
        assert_parity(c.spectrum()[2], ref["tot"])


def test_batch_graph_replay_with_fixed_buffers():
    """Steps written into the same device buffers each round replay a captured
    graph; results equal plain launches."""
    wls = small_jobs()[:3]
    ctxs = [rad.Context(wl.omega, wl.dirs, wl.ff_kind, wl.ff_width) for wl in wls]
    batch = rad.Batch(ctxs)
    bufs = []
    for wl in wls:
        st = wl.step(0)
        bufs.append([to_dev(st.r), to_dev(st.beta), to_dev(st.beta_dot), to_dev(st.w)])
    n0 = rad.kernel_launch_count()
    for s in range(6):
        steps = []
        for wl, b in zip(wls, bufs):
            st = wl.step(s)
            batch.sync()
            for dst, src in zip(b, (st.r, st.beta, st.beta_dot, st.w)):
                dst.copy_(torch.from_numpy(src))
            steps.append(rad.make_step(st.n, *b, st.t, st.dt))
        batch.accumulate(steps)
    batch.sync()
    # 7 kernels per round: the pre-pass, the four wide-call kernels (which return
    # at once for these compact jobs) and the two accumulate kernels
    assert rad.kernel_launch_count() - n0 == 6 * 7
    for wl, c in zip(wls, ctxs):
        ref = gpu_run(wl, range(6))
        for x, y in zip(ref.spectrum(), c.spectrum()):
            np.testing.assert_array_equal(x, y)


def test_checkpoint_resume_and_merge():
    wl = inputs.lwfa_bunch(n_particles=1200, n_omega=64, n_side=4, seed=31)
    full = gpu_run(wl, range(8))
    # checkpoint after 4 steps, resume in a fresh context
    a = gpu_run(wl, range(4))
    blob = a.state_export()
    b = rad.Context(wl.omega, wl.dirs, wl.ff_kind, wl.ff_width)
    b.state_import(blob)
    gpu_run(wl, range(4, 8), ctx=b)
    for x, y in zip(full.spectrum(), b.spectrum()):
        np.testing.assert_array_equal(x, y)
    # two "ranks" with disjoint halves of every step, merged on the host
    half = wl.n_particles // 2
    ranks = [rad.Context(wl.omega, wl.dirs, wl.ff_kind, wl.ff_width) for _ in range(2)]
    for s in range(8):
        st = wl.step(s)
        for k, sl in enumerate((slice(0, half), slice(half, None))):
            r = st.r.reshape(3, -1)[:, sl]
            b_ = st.beta.reshape(3, -1)[:, sl]
            bd = st.beta_dot.reshape(3, -1)[:, sl]
            ranks[k].accumulate(to_dev(r), to_dev(b_), to_dev(bd), to_dev(st.w[sl]), st.t, st.dt)
    ranks[0].state_merge(ranks[1].state_export())
    ref = spectra_grid(oracle_run(wl, range(8)), wl)
    assert_parity(ranks[0].spectrum()[2], ref["tot"])
    with pytest.raises(rad.RadError):
        other = rad.Context(wl.omega[:32], wl.dirs, wl.ff_kind, wl.ff_width)
        other.state_import(blob)


def test_tune_keeps_parity():
    wl = inputs.lwfa_bunch(n_particles=5000, n_omega=192, n_side=4, seed=41)
    ctx = rad.Context(wl.omega, wl.dirs, wl.ff_kind, wl.ff_width)
    tile = ctx.tune(5000)
    assert tile[0] in (0, 1, 2, 3, 4, 5, 7, 8, 9)  # 6 is the literal sum's own variant
    gpu_run(wl, range(5), ctx=ctx)
    ref = spectra_grid(oracle_run(wl, range(5)), wl)
    assert_parity(ctx.spectrum()[2], ref["tot"])


def test_batched_job_mix_at_full_size_sampled_bins():
    """The batched job mix at its full size, in the configuration the benchmark
    times (64 jobs of 1e3-1e6 macro-particles on 64-1024 frequencies x 16-1024
    directions, each round one persistent launch): two rounds of distinct steps,
    then 4 sampled bins of every job against the oracle under the per-bin gate."""
    specs = inputs.job_mix(64)
    wls = [s.workload() for s in specs]
    ctxs = [rad.Context(wl.omega, wl.dirs, wl.ff_kind, wl.ff_width) for wl in wls]
    batch = rad.Batch(ctxs)
    for r in range(2):
        data = [dev_steps(wl, r) for wl in wls]
        batch.accumulate([rad.make_step(st.n, *arrs, st.t, st.dt) for st, arrs in data])
        batch.sync()
    rng = np.random.default_rng(11)
    for j, (wl, ctx) in enumerate(zip(wls, ctxs)):
        got = dict(zip(("coh", "inc", "tot"), ctx.spectrum()))
        bins = [(int(rng.integers(0, wl.dirs.shape[0])), int(rng.integers(0, wl.omega.shape[0])))
                for _ in range(4)]
        ref = oracle_run(wl, range(2), bins).spectra()
        assert_sampled_bins(got, ref, bins, what=f"job {j}")
    batch.close()
    for c in ctxs:
        c.close()


@pytest.mark.parametrize("policy", [(0, 0), (1, 1), (2, 1_000_000), (3, 1_000_000), (4, 1_000_000)])
def test_server_results_equal_alone_and_in_the_mix(policy):
    """Jobs submitted at different times, steps fed incrementally, one slot fewer
    than jobs (admission waits); each result equals the standalone run, under
    every round policy (all ready jobs; one job per round in arrival order; least
    served first up to 1e6 updates per round, with and without aging; the oldest
    job with bounded backfill)."""
    wls = small_jobs()
    srv = rad.Server(hbm_budget=8 << 30, max_slots=3)
    srv.set_policy(*policy)
    ids = []
    fed = [0] * len(wls)
    for j, wl in enumerate(wls):
        ids.append(srv.submit(wl.omega, wl.dirs, wl.ff_kind, wl.ff_width, max_particles=wl.n_particles,
                              max_queued=2))
        time.sleep(0.01)
    deadline = time.time() + 120
    while min(fed) < 6 and time.time() < deadline:
        for j, wl in enumerate(wls):
            if fed[j] >= 6:
                continue
            st = wl.step(fed[j])
            step = rad.make_step(st.n, st.r, st.beta, st.beta_dot, st.w, st.t, st.dt)
            if srv.feed(ids[j], step) == rad.RAD_OK:
                fed[j] += 1
                if fed[j] == 6:
                    srv.finish(ids[j])
        time.sleep(0.001)
    assert min(fed) == 6
    for j, wl in enumerate(wls):
        coh, inc, tot, lat = srv.result(ids[j], wl.dirs.shape[0], wl.omega.shape[0], timeout=120)
        alone = gpu_run(wl, range(6)).spectrum()
        np.testing.assert_array_equal(tot, alone[2])
        np.testing.assert_array_equal(coh, alone[0])
        assert lat > 0
    st = srv.stats()
    assert st["completed"] == len(wls) and st["submitted"] == len(wls)
    srv.close()


def test_served_job_mix_sampled_bins():
    """Eight jobs of the serving mix at their full sizes (up to 1e6 particles
    and 1024 x 32^2 bins) submitted together to a server with four slots under
    the default policy, three steps each fed from device buffers: 4 sampled
    bins of every result against the oracle under the per-bin gate."""
    specs = inputs.job_mix(8, base_seed=5000, steps=(3, 3))
    wls = [s.workload() for s in specs]
    data = [[dev_steps(wl, s) for s in range(3)] for wl in wls]
    srv = rad.Server(hbm_budget=64 << 30, max_slots=4)
    ids = [srv.submit(wl.omega, wl.dirs, wl.ff_kind, wl.ff_width, max_particles=wl.n_particles,
                      max_queued=3) for wl in wls]
    for j in range(len(wls)):
        for st, arrs in data[j]:
            step = rad.make_step(st.n, *arrs, st.t, st.dt)
            deadline = time.time() + 60
            while srv.feed(ids[j], step) != rad.RAD_OK and time.time() < deadline:
                time.sleep(0.001)
        srv.finish(ids[j])
    rng = np.random.default_rng(12)
    for j, wl in enumerate(wls):
        coh, inc, tot, _ = srv.result(ids[j], wl.dirs.shape[0], wl.omega.shape[0], timeout=300)
        bins = [(int(rng.integers(0, wl.dirs.shape[0])), int(rng.integers(0, wl.omega.shape[0])))
                for _ in range(4)]
        ref = oracle_run(wl, range(3), bins).spectra()
        assert_sampled_bins({"coh": coh, "inc": inc, "tot": tot}, ref, bins, what=f"job {j}")
    srv.close()


def test_server_policy_arguments():
    srv = rad.Server(hbm_budget=1 << 30, max_slots=2)
    for bad in ((5, 10), (-1, 10), (1, 0), (2, -5), (3, 0), (4, 0)):
        with pytest.raises(rad.RadError):
            srv.set_policy(*bad)
    srv.set_policy(rad.SERVE_ALL, 0)
    srv.close()


def test_server_rejects_job_larger_than_budget():
    srv = rad.Server(hbm_budget=1 << 20, max_slots=1)
    with pytest.raises(rad.RadError):
        srv.submit(inputs.omega_log(1e14, 1e20, 1024), inputs.dirs_grid(0.01, 32, 32), max_particles=10 ** 6)
    srv.close()


def test_rad_log_reports_decisions_and_job_events():
    """RAD_LOG=2: the tuner's choice and each served job's admission and completion
    are printed to stderr (the level is read once per process, hence a subprocess)."""
    import os
    import subprocess
    import sys
    code = (
        "from paper_1802_03972_gb300 import rad, inputs\n"
        "wl = inputs.lwfa_bunch(n_particles=300, n_omega=64, n_side=2, seed=5)\n"
        "ctx = rad.Context(wl.omega, wl.dirs, wl.ff_kind, wl.ff_width)\n"
        "ctx.tune(wl.n_particles)\n"
        "srv = rad.Server(hbm_budget=1 << 30, max_slots=1)\n"
        "j = srv.submit(wl.omega, wl.dirs, wl.ff_kind, wl.ff_width, max_particles=wl.n_particles)\n"
        "st = wl.step(0)\n"
        "while srv.feed(j, rad.make_step(st.n, st.r, st.beta, st.beta_dot, st.w, st.t, st.dt)) != rad.RAD_OK:\n"
        "    pass\n"
        "srv.finish(j)\n"
        "srv.result(j, wl.dirs.shape[0], wl.omega.shape[0], timeout=60)\n"
        "srv.close()\n")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, RAD_LOG="2", PYTHONPATH=root)
    p = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300)
    assert p.returncode == 0, p.stderr[-2000:]
    err = p.stderr
    assert "[rad] tune: 64 omega x 4 directions" in err, err[-2000:]
    assert "admitted" in err and "done after" in err, err[-2000:]
