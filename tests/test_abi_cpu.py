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
