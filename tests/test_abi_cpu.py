"""CPU checks of the boundary: the library builds/loads and exports every
symbol the headers declare (no compute calls without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in ("rad.h", "rad_probe.h", "rad_selftest.h"):
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"\b(rad_\w+)\s*\(", src):
            names.add(m.group(1))
    return names


def test_library_exports_every_declared_symbol():
    from paper_1802_03972_gb300 import build, rad
    path = build.build()
    lib = ctypes.CDLL(path)
    decl = declared_symbols()
    assert decl, "no declarations parsed"
    missing = [n for n in sorted(decl) if not hasattr(lib, n)]
    assert not missing, missing
    assert decl == set(rad.EXPORTS), (decl ^ set(rad.EXPORTS))


def test_status_strings_and_launch_counter_without_gpu():
    from paper_1802_03972_gb300 import rad
    lib = rad.load()
    assert lib.rad_status_str(rad.RAD_EDATA) == b"invalid particle data"
    assert lib.rad_kernel_launch_count() >= 0


def test_struct_layouts_match_header():
    from paper_1802_03972_gb300 import rad
    assert ctypes.sizeof(rad.rad_ff) == 16
    assert ctypes.sizeof(rad.rad_tile) == 16
    assert ctypes.sizeof(rad.rad_step) == 56
    assert ctypes.sizeof(rad.rad_job_desc) == 56


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_1802_03972_gb300 import rad
    with pytest.raises(RuntimeError):
        rad._lib_saved = rad._lib
        try:
            rad._lib = None
            rad.load(str(tmp_path / "missing.so"))
        finally:
            rad._lib = rad._lib_saved


def build_c_client(out_dir):
    """Compiles tests/c_abi_client.c as C11 against include/rad.h and links it
    to the library; returns the executable's path."""
    import shutil
    import subprocess
    from paper_1802_03972_gb300 import build
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lib = build.build()
    libdir = os.path.dirname(lib)
    exe = os.path.join(str(out_dir), "c_abi_client")
    cmd = [cc, "-std=c11", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I", os.path.join(ROOT, "include"),
           os.path.join(ROOT, "tests", "c_abi_client.c"), "-o", exe, "-L", libdir, "-lrad",
           "-Wl,-rpath," + libdir]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


def test_header_compiles_as_c_and_client_links(tmp_path):
    import subprocess
    exe = build_c_client(tmp_path)
    r = subprocess.run([exe], capture_output=True, text=True)
    assert r.returncode == 2 and "usage" in r.stderr


def test_create_rejects_bad_arguments_before_touching_the_gpu():
    """rad_create validates its arguments on the host first, so every refusal
    below is RAD_EINVAL with no device present (and *out stays NULL)."""
    import numpy as np
    from paper_1802_03972_gb300 import rad
    lib = rad.load()
    om = np.array([1e14, 2e14])
    dirs = np.array([[0.0, 0.0, 1.0], [0.1, 0.0, 1.0]])
    big_om = np.full(65536, 1e15)
    big_dirs = np.tile([0.0, 0.0, 1.0], (32768, 1))
    ok_ff = rad.rad_ff(rad.FF_GAUSS, 0, 1e-7)
    cases = [
        (om, 0, dirs, 2, ok_ff, rad.PREC_MIXED),                      # no frequencies
        (om, 2, dirs, 0, ok_ff, rad.PREC_MIXED),                      # no directions
        (big_om, 65536, big_dirs, 32768, ok_ff, rad.PREC_MIXED),      # 2^31 bins
        (om, 2, dirs, 2, ok_ff, 7),                                   # unknown precision
        (om, 2, dirs, 2, rad.rad_ff(9, 0, 1e-7), rad.PREC_MIXED),     # unknown shape
        (om, 2, dirs, 2, rad.rad_ff(rad.FF_CIC, 0, -1.0), rad.PREC_MIXED),         # negative width
        (om, 2, dirs, 2, rad.rad_ff(rad.FF_CIC, 8, 1e-7), rad.PREC_MIXED),         # unknown flag
        (np.array([1e14, np.nan]), 2, dirs, 2, ok_ff, rad.PREC_MIXED),             # NaN frequency
        (np.array([1e14, -1.0]), 2, dirs, 2, ok_ff, rad.PREC_MIXED),               # negative frequency
        (om, 2, np.array([[0.0, 0.0, 1.0], [0.0, 0.0, 0.0]]), 2, ok_ff, rad.PREC_MIXED),  # zero direction
        (om, 2, dirs, 2, rad.rad_ff(rad.FF_CIC, rad.FF_LITERAL, 1e-7), rad.PREC_FP64),    # literal + FP64
        (om, 2, dirs, 2, rad.rad_ff(rad.FF_CIC, rad.FF_LITERAL | rad.FF_3D, 1e-7), rad.PREC_MIXED),
    ]
    for o, no, d, nd, ff, prec in cases:
        h = ctypes.c_void_p(1234)
        st = lib.rad_create(np.ascontiguousarray(o).ctypes.data, no, np.ascontiguousarray(d).ctypes.data,
                            nd, ff, prec, None, ctypes.byref(h))
        assert st == rad.RAD_EINVAL, (no, nd, prec)
        assert not h.value
    assert lib.rad_create(om.ctypes.data, 2, dirs.ctypes.data, 2, ok_ff, rad.PREC_MIXED, None, None) == rad.RAD_EINVAL


def test_every_entry_point_refuses_null_handles_without_a_gpu():
    """A NULL object or output pointer is RAD_EINVAL from every entry point
    (RAD_EINVAL = 1; rad_state_size gives 0; the destroy calls are no-ops)."""
    from paper_1802_03972_gb300 import rad
    lib = rad.load()
    t = rad.rad_tile()
    calls = {
        "rad_accumulate": (None, 1, None, None, None, None, 0.0, 1e-16),
        "rad_spectrum": (None, None, None, None),
        "rad_spectrum_ff": (None, rad.rad_ff(0, 0, 0.0), None, None, None),
        "rad_spectrum_literal": (None, None),
        "rad_spectrum_species": (None, None, 0, None, None, None),
        "rad_sync": (None,), "rad_reset": (None,), "rad_tune": (None, 1),
        "rad_get_tile": (None, ctypes.byref(t)), "rad_set_tile": (None, ctypes.byref(t)),
        "rad_state_export": (None, None, 0), "rad_state_import": (None, None, 0),
        "rad_state_merge": (None, None, 0), "rad_last_error": (None,),
        "rad_batch_create": (None, 0, None, None), "rad_batch_accumulate": (None, None),
        "rad_batch_sync": (None,), "rad_server_create": (1 << 30, 4, None, None),
        "rad_server_set_policy": (None, 2, 1), "rad_job_submit": (None, None, None),
        "rad_job_feed": (None, 0, None), "rad_job_finish": (None, 0), "rad_job_poll": (None, 0, None),
        "rad_job_result": (None, 0, 0.0, None, None, None, None), "rad_server_stats_get": (None, None),
        "rad_profile_enable": (None, 1), "rad_profile_read": (None, None, None, None),
        "rad_profile_clock": (None, None), "rad_selftest_wait": (1000000, None, None),
        "rad_selftest_stage1": (None, 1, None, None, None, None, 0.0, 1e-16, 0, None, None),
        "rad_selftest_phase": (None, 1, None, None, None, None),
        "rad_accumulate_static": (None, 0, None, 0, 0, None, None, None, None, 0.0, 1e-16, None, None),
        "rad_push_step": (None, 1, None, None, None, 0.0, 1e-16), "rad_push_flush": (None,),
    }
    for name, args in calls.items():
        assert getattr(lib, name)(*args) == rad.RAD_EINVAL, name
    assert lib.rad_state_size(None) == 0
    lib.rad_destroy(None)
    lib.rad_batch_destroy(None)
    lib.rad_server_destroy(None)


def test_every_header_compiles_as_pedantic_c11(tmp_path):
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "all_headers.c"
    src.write_text('#include "rad.h"\n#include "rad_probe.h"\n#include "rad_selftest.h"\n'
                   "int main(void) { return 0; }\n")
    r = subprocess.run([cc, "-std=c11", "-Wall", "-Wextra", "-Werror", "-pedantic", "-fsyntax-only",
                        "-I", os.path.join(ROOT, "include"), str(src)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_concurrent_build_waits_for_the_lock():
    """One process per rank may call build() at once: a second caller waits
    while another holds the build lock, then finds the library current."""
    import fcntl
    import subprocess
    import sys
    import time
    from paper_1802_03972_gb300 import build
    lib = build.build()
    root = os.path.dirname(os.path.dirname(os.path.abspath(build.__file__)))
    with open(os.path.join(build.OBJ, ".lock"), "w") as lock:
        fcntl.flock(lock, fcntl.LOCK_EX)
        child = subprocess.Popen(
            [sys.executable, "-c", "from paper_1802_03972_gb300 import build; print(build.build())"],
            cwd=root, stdout=subprocess.PIPE, text=True)
        time.sleep(1.0)
        assert child.poll() is None  # blocked on the lock
        fcntl.flock(lock, fcntl.LOCK_UN)
    out, _ = child.communicate(timeout=120)
    assert child.returncode == 0 and out.strip() == lib
