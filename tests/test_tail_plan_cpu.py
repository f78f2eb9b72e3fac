"""The fine-chunked tail plan (rad_impl.h: TailPlan, tail_plan) on the host: a
job that fills the GPU at least twice over cuts its last L = ceil(grid /
n_chunks) + 1 tiles into chunks of a quarter of the size, enough fine work for
every resident block to move on to it before the coarse items run out; small
jobs, FP32 variants and plans that would cover half the tiles or more are left
alone.  The plan is compiled from the library's own header with the host
compiler and checked against these rules and one worked case (the LWFA
workload: 1e5 particles, 256 tiles of 512 bins, 10 coarse chunks of 10752 on
304 resident blocks)."""
import math
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1802_03972_gb300", "csrc")
ALIGN = 256  # kChunkAlign


def _cuda_include():
    for base in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if base and os.path.exists(os.path.join(base, "include", "cuda_runtime.h")):
            return os.path.join(base, "include")
    nvcc = shutil.which("nvcc")
    if nvcc:
        inc = os.path.join(os.path.dirname(os.path.dirname(nvcc)), "include")
        if os.path.exists(os.path.join(inc, "cuda_runtime.h")):
            return inc
    return None


@pytest.fixture(scope="module")
def plan(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    inc = _cuda_include()
    if not cxx or not inc:
        pytest.skip("needs a host C++ compiler and the CUDA runtime headers")
    exe = str(tmp_path_factory.mktemp("tail") / "tail_plan_host")
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", os.path.join(ROOT, "include"), "-I", CSRC,
                    "-I", inc, os.path.join(ROOT, "tests", "tail_plan_host.cpp"), "-o", exe],
                   check=True, capture_output=True)

    def run(cases):
        text = "".join(" ".join(str(v) for v in c) + "\n" for c in cases)
        out = subprocess.run([exe], input=text, capture_output=True, text=True, check=True).stdout
        return [tuple(int(x) for x in line.split()) for line in out.splitlines()]
    return run


def expected(tc, n, n_tiles, ck, nc, grid):
    """The plan's rules restated."""
    if not tc or n <= 0 or n_tiles * nc < 2 * grid:
        return 0, 0, 0
    ckf = max(ALIGN, math.ceil(ck // 4 / ALIGN) * ALIGN)
    if ckf >= ck:
        return 0, 0, 0
    L = math.ceil(grid / nc) + 1
    if 2 * L > n_tiles:
        return 0, 0, 0
    return L, ckf, math.ceil(n / ckf)


def test_lwfa_workload_worked_case(plan):
    (tiles, ckf, ncf, items, fine), = plan([(1, 100000, 256, 10752, 10, 304, 512)])
    assert (tiles, ckf, ncf) == (32, 2816, 36)
    assert items == 224 * 10 + 32 * 36
    assert fine == 36 * 8 * 32 * 512


def test_plan_follows_its_rules(plan):
    cases = []
    for tc in (0, 1):
        for n in (1000, 20000, 100000, 1000000, 10000000):
            for n_tiles in (1, 8, 64, 256, 2048):
                for nc in (1, 2, 4, 10, 28, 76):
                    ck = math.ceil(math.ceil(n / nc) / ALIGN) * ALIGN
                    nc_real = math.ceil(n / ck)
                    for grid in (152, 304, 456):
                        cases.append((tc, n, n_tiles, ck, nc_real, grid, 512))
    got = plan(cases)
    assert len(got) == len(cases)
    for c, (tiles, ckf, ncf, items, fine) in zip(cases, got):
        tc, n, n_tiles, ck, nc, grid, bpt = c
        assert (tiles, ckf, ncf) == expected(tc, n, n_tiles, ck, nc, grid), c
        assert items == (n_tiles - tiles) * nc + tiles * ncf, c
        assert fine == ncf * 8 * tiles * bpt, c
        if tiles:
            assert ckf % ALIGN == 0 and ckf < ck, c
            assert tiles * nc >= grid, c          # fine work covers one coarse item per block
            assert 2 * tiles <= n_tiles, c
            assert (ncf - 1) * ckf < n <= ncf * ckf, c


def test_plan_is_off_where_it_cannot_help(plan):
    got = plan([
        (0, 100000, 256, 10752, 10, 304, 512),   # FP32 variant (and the literal sum)
        (1, 2000, 8, 256, 8, 304, 512),          # a job that does not fill the GPU twice
        (1, 262144, 3, 1024, 256, 304, 512),     # the fine tiles would be half the job or more
        (1, 1000, 4096, 256, 4, 304, 512),       # chunks already at the minimum
    ])
    assert [g[0] for g in got] == [0, 0, 0, 0]
