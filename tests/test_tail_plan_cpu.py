"""The fine-chunked tail plan (rad_impl.h: TailPlan, tail_plan) on the host.
A job that fills the GPU at least twice over cuts its last tiles finer, in two
levels: L0 = ceil(grid / n_chunks) + 1 tiles in chunks of a quarter of the
coarse chunk, enough fine work for every resident block to move on to it
before the coarse items run out, then the job's last L1 = ceil(grid / n1) + 1
tiles in chunks of a quarter of that (n1 chunks per tile), about one of these
items per block.  Small jobs, FP32 variants, chunks that cannot shrink below
one particle tile and plans that would cover half the tiles or more are left
alone (level 1 alone may drop out).  The plan is compiled from the library's
own header with the host compiler and checked against these rules and one
worked case (the LWFA workload: 1e5 particles, 256 tiles of 512 bins, 10
coarse chunks of 10752 on 304 resident blocks)."""
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
    """The plan's rules restated: ((L0, ck0, n0), (L1, ck1, n1))."""
    none = (0, 0, 0)
    if not tc or n <= 0 or n_tiles * nc < 2 * grid:
        return none, none
    levels, tiles = [], 0
    for level in range(2):
        ckf = max(ALIGN, math.ceil(ck // 4 / ALIGN) * ALIGN)
        if ckf >= ck:
            break
        ncf = math.ceil(n / ckf)
        L = math.ceil(grid / (nc if level == 0 else ncf)) + 1
        if 2 * (tiles + L) > n_tiles:
            break
        levels.append((L, ckf, ncf))
        tiles += L
        ck = ckf
    levels += [none] * (2 - len(levels))
    return tuple(levels)


def test_lwfa_workload_worked_case(plan):
    (t0, ck0, n0, t1, ck1, n1, items, fine, off1), = plan([(1, 100000, 256, 10752, 10, 304, 512)])
    assert (t0, ck0, n0) == (32, 2816, 36)
    assert (t1, ck1, n1) == (4, 768, 131)   # ceil(1e5 / 768) = 131, ceil(304 / 131) + 1 = 4
    assert items == 220 * 10 + 32 * 36 + 4 * 131
    assert off1 == 36 * 8 * 32 * 512
    assert fine == off1 + 131 * 8 * 4 * 512


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
    n_two = 0
    for c, (t0, ck0, n0, t1, ck1, n1, items, fine, off1) in zip(cases, got):
        tc, n, n_tiles, ck, nc, grid, bpt = c
        assert ((t0, ck0, n0), (t1, ck1, n1)) == expected(tc, n, n_tiles, ck, nc, grid), c
        assert items == (n_tiles - t0 - t1) * nc + t0 * n0 + t1 * n1, c
        assert off1 == n0 * 8 * t0 * bpt, c
        assert fine == off1 + n1 * 8 * t1 * bpt, c
        assert t0 or not t1, c                   # level 1 only after level 0
        prev = ck
        for tiles, ckf, ncf, cover in ((t0, ck0, n0, nc), (t1, ck1, n1, None)):
            if not tiles:
                continue
            assert ckf % ALIGN == 0 and ckf < prev, c
            assert (ncf - 1) * ckf < n <= ncf * ckf, c
            # level 0's work covers one coarse item per block, level 1 one of its own
            assert tiles * (cover or ncf) >= grid, c
            prev = ckf
        assert 2 * (t0 + t1) <= n_tiles, c
        # the serving engine's footprint bound on (tile, chunk) pairs
        assert t0 * n0 + t1 * n1 <= 6 * grid + 40 * nc + 12, c
        n_two += t1 > 0
    assert n_two > 20  # both levels are exercised


def test_plan_is_off_where_it_cannot_help(plan):
    got = plan([
        (0, 100000, 256, 10752, 10, 304, 512),   # FP32 variant (and the literal sum)
        (1, 2000, 8, 256, 8, 304, 512),          # a job that does not fill the GPU twice
        (1, 262144, 3, 1024, 256, 304, 512),     # the fine tiles would be half the job or more
        (1, 1000, 4096, 256, 4, 304, 512),       # chunks already at the minimum
    ])
    assert [g[0] for g in got] == [0, 0, 0, 0]
    assert [g[3] for g in got] == [0, 0, 0, 0]


def test_second_level_needs_room(plan):
    # level 0 only: its chunk is one particle tile already (1024 / 4 = 256)
    (g,) = plan([(1, 100000, 256, 1024, 98, 304, 512)])
    assert g[:3] == (5, 256, 391) and g[3] == 0
    # level 0 only: level 1 would take the job past half its tiles
    (g,) = plan([(1, 100000, 70, 10752, 10, 304, 512)])
    assert g[0] == 32 and g[3] == 0
