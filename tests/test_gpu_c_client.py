"""The library driven from plain C (tests/c_abi_client.c, nothing but
include/rad.h): host particle arrays in, host spectra out.  Its spectra must
match the FP64 oracle within the parity tolerance, and equal bit for bit what
the Python binding gets from the same calls."""
import struct
import subprocess

import numpy as np
import pytest

from gpu_util import assert_parity, oracle_run, spectra_grid
from paper_1802_03972_gb300 import inputs
from test_abi_cpu import build_c_client

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1802_03972_gb300 import build as _build  # noqa: E402

_build.build()
from paper_1802_03972_gb300 import rad  # noqa: E402


def write_job(path, wl, steps):
    n = wl.n_particles
    with open(path, "wb") as f:
        f.write(struct.pack("=iiiiqd", wl.omega.size, wl.dirs.shape[0], len(steps), wl.ff_kind, n,
                            wl.ff_width))
        f.write(np.ascontiguousarray(wl.omega, dtype=np.float64).tobytes())
        f.write(np.ascontiguousarray(wl.dirs, dtype=np.float64).tobytes())
        for s in steps:
            st = wl.step(s)
            f.write(struct.pack("=dd", st.t, st.dt))
            for a in (st.r, st.beta, st.beta_dot, st.w):
                f.write(np.ascontiguousarray(a, dtype=np.float64).ravel().tobytes())


def test_c_client_matches_oracle_and_binding(tmp_path):
    wl = inputs.lwfa_bunch(n_particles=1300, n_omega=96, n_side=4, seed=71)
    steps = range(5)
    exe = build_c_client(tmp_path)
    job, out = tmp_path / "job.bin", tmp_path / "spectra.bin"
    write_job(job, wl, steps)
    r = subprocess.run([exe, str(job), str(out)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    got = np.fromfile(out, dtype=np.float64).reshape(3, wl.dirs.shape[0], wl.omega.size)
    ref = spectra_grid(oracle_run(wl, steps), wl)
    for k, g in zip(("coh", "inc", "tot"), got):
        assert_parity(g, ref[k], what=k)
    ctx = rad.Context(wl.omega, wl.dirs, wl.ff_kind, wl.ff_width)
    for s in steps:
        st = wl.step(s)
        ctx.accumulate(st.r, st.beta, st.beta_dot, st.w, st.t, st.dt)
    for a, b in zip(got, ctx.spectrum()):
        np.testing.assert_array_equal(a, b)
