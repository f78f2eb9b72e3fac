"""Failures made on the host, and what the library must do about them.

* a job with invalid particles (NaN position, |beta| > 1) inside a batch or a
  served mix: that job reports RAD_EDATA once and its spectrum covers its valid
  particles; every other job stays bitwise equal to running alone;
* a server destroyed with jobs admitted, waiting and part-fed: it returns
  promptly and the device stays usable;
* a bounded device wait that nothing completes (rad_selftest_wait): it gives up
  after its limit and reports it, and the context keeps working.
Nothing here faults or hangs a GPU."""
import threading
import time

import numpy as np
import pytest

from gpu_util import assert_parity, gpu_run, oracle_run, spectra_grid, to_dev
from paper_1802_03972_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1802_03972_gb300 import build as _build  # noqa: E402

_build.build()
from paper_1802_03972_gb300 import rad  # noqa: E402


def jobs():
    specs = [inputs.JobSpec(9000 + j, n, no, ns, 4, 100.0, 300.0, 2e-6)
             for j, (n, no, ns) in enumerate([(900, 64, 4), (500, 128, 2), (1300, 32, 4)])]
    return [s.workload() for s in specs]


def poisoned(st):
    """The step's arrays with two invalid particles appended (NaN position, |beta| = 1.5)."""
    r = np.concatenate([st.r.reshape(3, -1), np.array([[np.nan, 0.0], [0.0, 0.0], [0.0, 0.0]])], 1)
    b = np.concatenate([st.beta.reshape(3, -1), np.array([[0.0, 0.0], [0.0, 0.0], [0.5, 1.5]])], 1)
    bd = np.concatenate([st.beta_dot.reshape(3, -1), np.ones((3, 2)) * 1e13], 1)
    w = np.concatenate([st.w, [10.0, 10.0]])
    return [a.ravel() for a in (r, b, bd)] + [w]


def test_bad_job_in_a_batch():
    wls = jobs()
    alone = [gpu_run(wl, range(4)) for wl in wls]
    ctxs = [rad.Context(wl.omega, wl.dirs, wl.ff_kind, wl.ff_width) for wl in wls]
    batch = rad.Batch(ctxs)
    keep = []
    for s in range(4):
        steps = []
        for j, wl in enumerate(wls):
            st = wl.step(s)
            arrs = [to_dev(a) for a in (poisoned(st) if j == 1 else (st.r, st.beta, st.beta_dot, st.w))]
            keep.append(arrs)
            steps.append(rad.make_step(int(arrs[3].shape[0]), *arrs, st.t, st.dt))
        batch.accumulate(steps)
    batch.sync()
    for j in (0, 2):
        for x, y in zip(alone[j].spectrum(), ctxs[j].spectrum()):
            np.testing.assert_array_equal(x, y)
    with pytest.raises(rad.RadError) as ei:
        ctxs[1].spectrum()
    assert ei.value.status == rad.RAD_EDATA
    ref = spectra_grid(oracle_run(wls[1], range(4)), wls[1])  # the valid particles only
    assert_parity(ctxs[1].spectrum()[2], ref["tot"])  # reported once


def test_bad_job_in_a_served_mix():
    wls = jobs()
    srv = rad.Server(hbm_budget=4 << 30, max_slots=2)  # one job waits for a slot
    ids = [srv.submit(wl.omega, wl.dirs, wl.ff_kind, wl.ff_width,
                      max_particles=wl.n_particles + 2, max_queued=2) for wl in wls]
    fed = [0] * len(wls)
    deadline = time.time() + 120
    while min(fed) < 4 and time.time() < deadline:
        for j, wl in enumerate(wls):
            if fed[j] == 4:
                continue
            st = wl.step(fed[j])
            arrs = poisoned(st) if j == 1 else [st.r, st.beta, st.beta_dot, st.w]
            if srv.feed(ids[j], rad.make_step(arrs[3].shape[0], *arrs, st.t, st.dt)) == rad.RAD_OK:
                fed[j] += 1
                if fed[j] == 4:
                    srv.finish(ids[j])
        time.sleep(0.001)
    assert min(fed) == 4
    for j, wl in enumerate(wls):
        nd, no = wl.dirs.shape[0], wl.omega.shape[0]
        if j == 1:
            with pytest.raises(rad.RadError) as ei:
                srv.result(ids[j], nd, no, timeout=120)
            assert ei.value.status == rad.RAD_EDATA
        else:
            tot = srv.result(ids[j], nd, no, timeout=120)[2]
            np.testing.assert_array_equal(tot, gpu_run(wl, range(4)).spectrum()[2])
    srv.close()


def test_bad_job_result_keeps_its_valid_spectrum():
    wl = jobs()[0]
    srv = rad.Server(hbm_budget=1 << 30, max_slots=1)
    jid = srv.submit(wl.omega, wl.dirs, wl.ff_kind, wl.ff_width, max_particles=wl.n_particles + 2)
    for s in range(4):
        st = wl.step(s)
        step = rad.make_step(wl.n_particles + 2, *poisoned(st), st.t, st.dt)
        while srv.feed(jid, step) != rad.RAD_OK:
            time.sleep(0.001)
    srv.finish(jid)
    tot = srv.result(jid, wl.dirs.shape[0], wl.omega.shape[0], timeout=120, accept_edata=True)[2]
    ref = spectra_grid(oracle_run(wl, range(4)), wl)
    assert_parity(tot, ref["tot"])
    srv.close()


def test_server_shutdown_with_jobs_in_flight():
    wls = jobs()
    srv = rad.Server(hbm_budget=4 << 30, max_slots=1)
    ids = [srv.submit(wl.omega, wl.dirs, wl.ff_kind, wl.ff_width, max_particles=wl.n_particles,
                      max_queued=2) for wl in wls]
    st = wls[0].step(0)
    assert srv.feed(ids[0], rad.make_step(st.n, st.r, st.beta, st.beta_dot, st.w, st.t, st.dt)) in (
        rad.RAD_OK, rad.RAD_EBUSY)
    done = threading.Event()
    t = threading.Thread(target=lambda: (srv.close(), done.set()), daemon=True)
    t.start()
    assert done.wait(60), "rad_server_destroy did not return"
    # the device is still usable
    ctx = gpu_run(wls[2], range(2))
    ref = spectra_grid(oracle_run(wls[2], range(2)), wls[2])
    assert_parity(ctx.spectrum()[2], ref["tot"])


def test_bounded_wait_gives_up_and_the_context_keeps_working():
    wl = jobs()[0]
    ctx = gpu_run(wl, range(2))
    timed_out, waited = rad.selftest_wait(50_000_000)  # 50 ms on an mbarrier nothing completes
    assert timed_out
    assert 0.045 <= waited <= 5.0, waited
    gpu_run(wl, range(2, 4), ctx=ctx)
    ref = spectra_grid(oracle_run(wl, range(4)), wl)
    assert_parity(ctx.spectrum()[2], ref["tot"])
