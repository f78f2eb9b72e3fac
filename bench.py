#!/usr/bin/env python3
"""Benchmark of the far-field radiation sum: amplitude updates per second.

One step = one rad_accumulate call over one time step of the LWFA-shaped bunch
(1e5 macro-particles, 512 log-spaced frequencies 1e14..1e20 rad/s, 16 x 16
directions within +-10 mrad, Gaussian form factor sigma = 0.1 um): 1.34e10
amplitude updates (particle x omega x n).  Inputs are synthetic, resident in HBM
before the timed region, and distinct per step (a ring of 64 steps x 8 MB =
512 MB, larger than L2).  Prints one JSON line.

  python bench.py [--steps K] [--warmup W] [--gpus N] [--impl ours|reference]

--impl reference times the FP64 CPU oracle on the host cores (a bounded sample
of bins per step); N > 1 under torchrun runs one independent job per rank.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "amplitude updates/s (particle×ω×n×step) at ≤1e-5 rel err; p50/p99 job latency"
UNIT = "updates/s"
SM_MAX_MHZ = 2070.0
MUFU_PER_CLK_SM = 16.0   # sin/cos lane-ops per clock per SM (measured by rad_probe_peaks)
MUFU_PER_UPDATE = 2.0    # one sin and one cos per (particle, omega, n)
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "accumulate_lwfa_traffic.json")
VARIANT_NAMES = {0: "FP32 FMA, 256 threads x 2 omega, 3 CTAs/SM",
                 1: "FP32 FMA, 256 threads x 4 omega, 2 CTAs/SM",
                 2: "FP32 FMA, 128 threads x 2 omega, 6 CTAs/SM",
                 3: "tensor-core accumulation (mma.sync TF32 hi/lo), 256 threads, 3 CTAs/SM",
                 4: "tensor-core accumulation (mma.sync TF32 hi/lo), 256 threads, 4 CTAs/SM",
                 5: "FP32 FMA, 256 threads x 2 omega, 4 CTAs/SM",
                 7: "tensor-core accumulation (mma.sync TF32 hi/lo), 256 threads, 3 CTAs/SM, "
                    "two frequency passes per staged particle tile",
                 8: "tensor-core accumulation (mma.sync TF32 hi/lo), 256 threads x 2 omega "
                    "(64 per warp), 2 CTAs/SM",
                 9: "tensor-core accumulation (mma.sync TF32 hi/lo), 256 threads x 2 omega "
                    "(64 per warp), 2 CTAs/SM, phase cross terms by mma.sync"}
# The accumulate kernel's sources: the kernel file and the headers its device code comes from.
KERNEL_SRC = [os.path.join(ROOT, "paper_1802_03972_gb300", "csrc", f)
              for f in ("rad_accumulate.cu", "rad_stage.cuh", "rad_device.cuh", "rad_impl.h")]


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=400)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--ring", type=int, default=64)
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-fp64", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-tune", action="store_true", help="keep the default tile instead of rad_tune")
    p.add_argument("--tile", default=None, help="fixed tile 'variant,omega_tile,chunk' (no tuning)")
    p.add_argument("--no-batch", action="store_true")
    p.add_argument("--batch-rounds", type=int, default=3)
    p.add_argument("--no-serve", action="store_true")
    p.add_argument("--serve-jobs", type=int, default=12)
    p.add_argument("--serve-steps", default="50,500",
                   help="range of steps per job of the load-relative serving leg")
    p.add_argument("--no-fifo-run", action="store_true",
                   help="skip the measured one-job-at-a-time FIFO run of the serving leg")
    p.add_argument("--no-insitu", action="store_true",
                   help="skip the in-situ-scale leg (1e7 particles, 1024 x 32^2 bins)")
    p.add_argument("--no-horizon", action="store_true",
                   help="skip the 256-step accuracy leg")
    p.add_argument("--no-helix", action="store_true",
                   help="skip the tiny helix leg (1000 small steps, mixed, FP64 and oracle)")
    p.add_argument("--wide-only", action="store_true",
                   help="profiling aid: run only the wide-bunch leg for --steps steps (after one "
                        "warm-up call) and print its figures")
    p.add_argument("--serve-load", type=float, default=0.7,
                   help="arrival rate as a fraction of measured capacity")
    p.add_argument("--no-modes", action="store_true",
                   help="skip the literal-sum, in-situ coupling and 3-D readout timings")
    p.add_argument("--serve-policy", default=None,
                   help="round policy 'P,ROUND_UPDATES' of the serving legs (0 all, 1 oldest, "
                        "2 least served, 3 least served with aging, 4 oldest with bounded "
                        "backfill; default: the library's)")
    p.add_argument("--serve-rate", type=float, default=None,
                   help="fixed arrival rate (jobs/s) instead of --serve-load")
    p.add_argument("--peaks", action="store_true", help="also run the pipe-throughput probe")
    return p.parse_args()


def config(wl, extra=None):
    c = {"workload": "lwfa_bunch (1e5 macro-particles, 512 log omega 1e14-1e20 rad/s, "
                     "16x16 directions +-10 mrad, Gaussian form factor 0.1 um)",
         "n_particles": wl.n_particles, "n_omega": int(wl.omega.shape[0]),
         "n_dir": int(wl.dirs.shape[0]), "updates_per_step": wl.updates_per_step(),
         "l2": "inputs larger than L2: distinct per-step particle arrays, ring of 64 x 8 MB"}
    if extra:
        c.update(extra)
    return c


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def kernel_hash() -> str:
    """Hash of the kernel's code: its sources with comments and blank space
    removed, so that editing a comment does not orphan a capture."""
    import re
    h = hashlib.sha256()
    for f in KERNEL_SRC:
        src = open(f, encoding="utf-8").read()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        h.update(" ".join(src.split()).encode())
    return h.hexdigest()[:16]


def traffic_per_launch(updates_per_step: int, tile):
    """DRAM bytes per accumulate launch from the committed ncu summary, scaled to this
    launch's updates; None when the kernel source or the tile changed since the capture."""
    try:
        captures = json.load(open(TRAFFIC_FILE))["captures"]
    except (OSError, ValueError, KeyError):
        return None
    sha = kernel_hash()
    for t in captures:
        if t.get("kernel_sha") == sha and list(t.get("tile", [])) == list(tile):
            return t["dram_bytes_per_launch"] * updates_per_step / t["updates_per_launch"]
    return None


def cpu_oracle_rate(wl, n_bins: int, target_s: float):
    """Oracle (as it stands) on n_bins sampled bins x all particles, steps until
    about target_s of CPU work: returns (updates/s, threads, description, steps)."""
    import numpy as np

    import oracle
    rng = np.random.default_rng(123)
    bins = [(int(rng.integers(0, wl.dirs.shape[0])), int(rng.integers(0, wl.omega.shape[0])))
            for _ in range(n_bins)]
    bo, bd = oracle.grid_bins(wl.omega, wl.dirs, bins)
    acc = oracle.Accumulator(bo, bd, wl.ff_kind, wl.ff_width)
    st = wl.step(0)
    t0 = time.perf_counter()
    acc.accumulate(st.r, st.beta, st.beta_dot, st.w, st.t, st.dt)
    t1 = time.perf_counter() - t0
    steps = max(1, min(200, int(round(target_s / max(t1, 1e-6)))))
    data = [wl.step(s) for s in range(1, steps + 1)]
    t0 = time.perf_counter()
    for st in data:
        acc.accumulate(st.r, st.beta, st.beta_dot, st.w, st.t, st.dt)
    el = time.perf_counter() - t0
    upd = n_bins * wl.n_particles * steps
    desc = (f"{n_bins} sampled (direction, omega) bins x {wl.n_particles} macro-particles x "
            f"{steps} steps = {upd:.3g} updates in {el:.1f} s")
    return upd / el, oracle.num_threads(), desc, steps


def reference_arm(args, wl):
    """FP64 CPU oracle, a bounded sample of bins per step, rank 0 only."""
    import numpy as np

    import oracle
    oracle.build()
    rng = np.random.default_rng(7)
    # bins per step so that one step takes ~0.3 s
    probe = [(int(rng.integers(0, 256)), int(rng.integers(0, 512))) for _ in range(16)]
    bo, bd = oracle.grid_bins(wl.omega, wl.dirs, probe)
    acc = oracle.Accumulator(bo, bd, wl.ff_kind, wl.ff_width)
    st = wl.step(0)
    t0 = time.perf_counter()
    acc.accumulate(st.r, st.beta, st.beta_dot, st.w, st.t, st.dt)
    per_bin = (time.perf_counter() - t0) / 16
    n_bins = int(max(16, min(4096, 0.3 / max(per_bin, 1e-9))))
    bins = [(int(rng.integers(0, 256)), int(rng.integers(0, 512))) for _ in range(n_bins)]
    bo, bd = oracle.grid_bins(wl.omega, wl.dirs, bins)
    acc = oracle.Accumulator(bo, bd, wl.ff_kind, wl.ff_width)
    data = [wl.step(s % 64) for s in range(min(64, args.steps + args.warmup))]
    for s in range(args.warmup):
        st = data[s % len(data)]
        acc.accumulate(st.r, st.beta, st.beta_dot, st.w, st.t, st.dt)
    t0 = time.perf_counter()
    for s in range(args.steps):
        st = data[(args.warmup + s) % len(data)]
        acc.accumulate(st.r, st.beta, st.beta_dot, st.w, st.t, st.dt)
    el = time.perf_counter() - t0
    upd = n_bins * wl.n_particles * args.steps
    value = upd / el
    sample = (f"each step: {n_bins} sampled (direction, omega) bins x {wl.n_particles} "
              f"macro-particles of the LWFA-shaped bunch")
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": config(wl, {"bins_per_step": n_bins}),
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(),
                            "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def modes_leg(wl, ring_dev, steps_host, upd: int, n_steps: int = 20):
    """Throughput of the other accumulation modes on the headline workload:
    the paper's literal sum (FF_LITERAL), in-situ coupling (push_step: beta_dot
    differenced on the device), the readout with the direction-dependent 3-D
    box form factor and the readout of two species with different shapes, each
    timed with CUDA events on the current stream."""
    import torch

    from paper_1802_03972_gb300 import rad
    ring = len(ring_dev)
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    out = {}
    lit = rad.Context(wl.omega, wl.dirs, wl.ff_kind, wl.ff_width, ff_flags=rad.FF_LITERAL)
    lit.accumulate(*ring_dev[0], steps_host[0].t, steps_host[0].dt)
    lit.sync()
    a, b = ev(), ev()
    a.record()
    for k in range(n_steps):
        st = steps_host[k % ring]
        lit.accumulate(*ring_dev[k % ring], st.t, st.dt)
    b.record()
    torch.cuda.synchronize()
    out["literal_sum"] = {"value": n_steps * upd / (a.elapsed_time(b) / 1e3), "unit": UNIT,
                          "steps": n_steps, "tile": list(lit.get_tile())}
    push = rad.Context(wl.omega, wl.dirs, wl.ff_kind, wl.ff_width)
    a, b = ev(), ev()
    a.record()
    for k in range(n_steps):
        st = steps_host[k % ring]
        r, beta, _, w = ring_dev[k % ring]
        push.push_step(r, beta, w, st.t, st.dt)
    push.push_flush()
    b.record()
    torch.cuda.synchronize()
    out["push_coupling"] = {"value": n_steps * upd / (a.elapsed_time(b) / 1e3), "unit": UNIT,
                            "steps": n_steps}
    bufs = [torch.empty((wl.dirs.shape[0], wl.omega.shape[0]), dtype=torch.float64, device="cuda")
            for _ in range(3)]
    times = {}
    for name, ff in (("readout_1d_ms", (rad.FF_CIC, 0.1e-6)), ("readout_3d_ms", (rad.FF_CIC, 0.1e-6, rad.FF_3D))):
        push.spectrum(ff=ff, out=bufs)
        a, b = ev(), ev()
        a.record()
        for _ in range(10):
            push.spectrum(ff=ff, out=bufs)
        b.record()
        torch.cuda.synchronize()
        times[name] = a.elapsed_time(b) / 10
    species = ([push, lit], [(rad.FF_GAUSS, 0.1e-6), (rad.FF_CIC, 0.1e-6, rad.FF_3D)])
    rad.spectrum_species(*species, out=bufs)
    a, b = ev(), ev()
    a.record()
    for _ in range(10):
        rad.spectrum_species(*species, out=bufs)
    b.record()
    torch.cuda.synchronize()
    times["readout_2_species_ms"] = a.elapsed_time(b) / 10
    out["readout"] = dict(times, bins=int(wl.dirs.shape[0] * wl.omega.shape[0]))
    push.close()
    lit.close()
    return out


def wide_leg(wl, tile, n_steps: int = 10):
    """The headline workload's grids with its bunch stretched to 2 mm along z
    (z uniform over +-1 mm, the rest as generated): about 50 times the fast
    phase range about one reference point, as when one call holds a whole
    domain (Sec. 3.3).  The call is sorted and its tiles rotated per group;
    timed like the headline, in the same tile."""
    import numpy as np
    import torch

    from paper_1802_03972_gb300 import rad
    rng = np.random.default_rng(12)
    n = wl.n_particles
    ring = []
    for s in range(n_steps):
        st = wl.step(s)
        r = st.r.reshape(3, n).copy()
        r[2] = rng.uniform(-1e-3, 1e-3, n) + 299792458.0 * st.t
        ring.append(([torch.from_numpy(np.ascontiguousarray(a)).cuda()
                      for a in (r.ravel(), st.beta, st.beta_dot, st.w)], st.t, st.dt))
    ctx = rad.Context(wl.omega, wl.dirs, wl.ff_kind, wl.ff_width)
    ctx.set_tile(*tile)
    ctx.accumulate(*ring[0][0], ring[0][1], ring[0][2])
    ctx.sync()
    ctx.profile(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for d, t_, dt in ring:
        ctx.accumulate(*d, t_, dt)
    e1.record()
    torch.cuda.synchronize()
    pre_ms, acc_ms, calls = ctx.profile_read()
    el = e0.elapsed_time(e1) / 1e3
    ctx.close()
    upd = wl.updates_per_step()
    return {"workload": "headline grids, 1e5 macro-particles with z uniform over +-1 mm",
            "value": n_steps * upd / el, "unit": UNIT, "steps": n_steps, "tile": list(tile),
            "prepass_and_sort_ms_per_step": pre_ms / max(calls, 1),
            "accumulate_ms_per_step": acc_ms / max(calls, 1)}


def batch_leg(rounds: int, n_jobs: int = 64, specs=None, mix: str = "batched job mix"):
    """n_jobs independent jobs (default: the batched job mix) advanced one step per
    round in one persistent launch, CUDA-graph replayed; against the same jobs
    launched one context at a time.  Returns a dict for the JSON line."""
    import torch

    from paper_1802_03972_gb300 import inputs, rad
    specs = specs if specs is not None else inputs.job_mix(n_jobs)
    n_jobs = len(specs)
    wls = [s.workload() for s in specs]
    dev, ctxs = [], []
    for wl in wls:
        st = wl.step(0)
        dev.append([torch.from_numpy(a).cuda() for a in (st.r, st.beta, st.beta_dot, st.w)])
        ctxs.append(rad.Context(wl.omega, wl.dirs, wl.ff_kind, wl.ff_width))
    upd = sum(s.updates_per_step() for s in specs)
    batch = rad.Batch(ctxs)

    def steps(r):
        return [rad.make_step(wl.n_particles, *d, r * wl.dt, wl.dt) for wl, d in zip(wls, dev)]

    batch.accumulate(steps(0))  # captures the graph
    batch.sync()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = rad.kernel_launch_count()
    e0.record()
    for r in range(1, rounds + 1):
        batch.accumulate(steps(r))
    e1.record()
    torch.cuda.synchronize()
    l_batch = (rad.kernel_launch_count() - l0) / rounds
    t_batch = e0.elapsed_time(e1) / 1e3 / rounds
    # unbatched: one launch pair per job per round, in submission order
    for c, wl, d in zip(ctxs, wls, dev):  # warm: each context's buffers exist
        c.accumulate(*d, wl.dt, wl.dt)
    torch.cuda.synchronize()
    l0 = rad.kernel_launch_count()
    e0.record()
    for r in range(rounds):
        for c, wl, d in zip(ctxs, wls, dev):
            c.accumulate(*d, (r + 2) * wl.dt, wl.dt)
    e1.record()
    torch.cuda.synchronize()
    l_seq = (rad.kernel_launch_count() - l0) / rounds
    t_seq = e0.elapsed_time(e1) / 1e3 / rounds
    batch.close()
    for c in ctxs:
        c.close()
    return {"mix": mix, "jobs": n_jobs, "updates_per_round": upd, "rounds": rounds,
            "value": upd / t_batch, "unit": UNIT, "ms_per_round": 1e3 * t_batch,
            "unbatched_value": upd / t_seq, "unbatched_ms_per_round": 1e3 * t_seq,
            "batched_over_unbatched": t_seq / t_batch, "launches_per_round": l_batch,
            "unbatched_launches_per_round": l_seq, "graph_replay": True}


# Per-bin gate of the parity tests: |I - I_ref| <= BIN_REL I_ref + 2 BIN_AMP
# sqrt(I_ref M) + BIN_AMP^2 M, M = the direction's largest I_ref (a relative
# error of the bin's own amplitude plus an absolute amplitude error of BIN_AMP
# times the direction's largest amplitude).
BIN_REL, BIN_AMP = 1e-5, 2e-6


def error_stats(got, ref, floor: float = 1e-6) -> dict:
    """Accuracy of a [rows][n_omega] spectrum against a reference: the largest
    per-direction relative 2-norm error ("row"); the largest ratio of a bin's
    error to its per-bin allowance ("bin_excess", <= 1 passes the per-bin gate);
    and the per-bin relative error (max and 99th percentile) over the bins whose
    reference is at least `floor` times its direction's maximum (spectral nulls
    have relative error ~1 at any precision and are left out)."""
    import numpy as np
    got = np.asarray(got, dtype=np.float64).reshape(np.shape(ref))
    ref = np.asarray(ref, dtype=np.float64)
    row, rels, excess = 0.0, [], 0.0
    for g, r in zip(got, ref):
        nr = np.linalg.norm(r)
        if nr == 0.0:
            row = max(row, 0.0 if np.linalg.norm(g) == 0.0 else math.inf)
            continue
        row = max(row, float(np.linalg.norm(g - r) / nr))
        m = np.abs(r).max()
        allowed = BIN_REL * np.abs(r) + 2.0 * BIN_AMP * np.sqrt(np.abs(r) * m) + BIN_AMP ** 2 * m
        excess = max(excess, float(np.max(np.abs(g - r) / allowed)))
        keep = np.abs(r) >= floor * m
        rels.append(np.abs(g[keep] - r[keep]) / np.abs(r[keep]))
    rel = np.concatenate(rels) if rels else np.zeros(0)
    return {"row": row, "bin_excess": excess, "bin_max": float(rel.max()) if rel.size else 0.0,
            "bin_p99": float(np.percentile(rel, 99)) if rel.size else 0.0, "bins": int(rel.size)}


def fifo_latencies(arrivals, work, rate: float):
    """Arrival-to-result latencies of one-job-at-a-time FIFO service at `rate` updates/s."""
    import numpy as np
    free, lat = 0.0, []
    for a, u in zip(arrivals, work):
        free = max(free, a) + u / rate
        lat.append(free - a)
    lat = np.array(lat)
    return {"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "rate": rate}


def fifo_run(specs, wls, dev, arrivals) -> dict:
    """One job at a time in arrival order, unbatched, through rad.Context: a job
    starts when it has arrived and the previous one is done, runs all its steps
    and reads its spectrum to the host.  Returns p50/p99 of arrival-to-result
    latency (measured) and the window's throughput."""
    import numpy as np
    import torch

    from paper_1802_03972_gb300 import rad
    order = np.argsort(arrivals, kind="stable")
    lat = np.zeros(len(specs))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for j in order:
        now = time.perf_counter() - t0
        if now < arrivals[j]:
            time.sleep(arrivals[j] - now)
        wl = wls[j]
        ctx = rad.Context(wl.omega, wl.dirs, wl.ff_kind, wl.ff_width)
        for s in range(specs[j].n_steps):
            ctx.accumulate(*dev[j], s * wl.dt, wl.dt)
        ctx.spectrum()
        ctx.close()
        lat[j] = time.perf_counter() - t0 - arrivals[j]
    makespan = time.perf_counter() - t0
    work = sum(s.updates_per_step() * s.n_steps for s in specs)
    return {"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean()), "value": work / makespan, "unit": UNIT,
            "makespan_s": makespan, "measured": True}


def serve_leg(n_jobs: int, load: float, rate: float | None, steps_range=(5, 20), seed: int = 5,
              cap: float = 1.6e12, fifo_rates=None, policy=None, run_fifo: bool = False):
    """Continuous batching: Poisson arrivals of the batched job mix (steps per job
    in steps_range), each job fed step by step from device buffers; p50/p99 of
    arrival-to-result latency and the throughput of the window.  `cap` is the
    measured single-GPU rate the load is relative to.  run_fifo: also run the
    same arrivals one job at a time (unbatched FIFO, measured).  `fifo_rates`
    names single-job rates whose FIFO latencies over the same arrivals are
    computed from the rates (a model, labelled as such)."""
    import numpy as np
    import torch

    from paper_1802_03972_gb300 import inputs, rad
    specs = inputs.job_mix(n_jobs, base_seed=5000, steps=steps_range)
    wls = [s.workload() for s in specs]
    work = [s.updates_per_step() * s.n_steps for s in specs]
    dev = []
    for wl in wls:
        st = wl.step(0)
        dev.append([torch.from_numpy(a).cuda() for a in (st.r, st.beta, st.beta_dot, st.w)])
    lam = rate if rate else load * cap / float(np.mean(work))
    rng = np.random.default_rng(seed)
    arrivals = np.cumsum(rng.exponential(1.0 / lam, n_jobs))
    srv = rad.Server(hbm_budget=150 << 30, max_slots=64)
    if policy:
        srv.set_policy(*policy)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ids, fed, done, lat = [None] * n_jobs, [0] * n_jobs, [False] * n_jobs, [None] * n_jobs
    nxt = 0
    while not all(done):
        now = time.perf_counter() - t0
        busy = False
        while nxt < n_jobs and arrivals[nxt] <= now:
            wl = wls[nxt]
            ids[nxt] = srv.submit(wl.omega, wl.dirs, wl.ff_kind, wl.ff_width,
                                  max_particles=wl.n_particles, max_queued=2)
            nxt += 1
            busy = True
        for j in range(nxt):
            if done[j]:
                continue
            wl = wls[j]
            if fed[j] < specs[j].n_steps:
                st = rad.make_step(wl.n_particles, *dev[j], fed[j] * wl.dt, wl.dt)
                if srv.feed(ids[j], st) == rad.RAD_OK:
                    fed[j] += 1
                    busy = True
                    if fed[j] == specs[j].n_steps:
                        srv.finish(ids[j])
            elif srv.poll(ids[j]):
                *_, lat[j] = srv.result(ids[j], wl.dirs.shape[0], wl.omega.shape[0])
                done[j] = True
                busy = True
        if not busy:
            time.sleep(0.0005)
    makespan = time.perf_counter() - t0
    stats = srv.stats()
    srv.close()
    lat = np.array(lat)
    out = {"jobs": n_jobs, "arrival_rate_per_s": lam, "load": load if not rate else None,
           "steps_per_job": list(steps_range), "p50_s": float(np.percentile(lat, 50)),
           "p99_s": float(np.percentile(lat, 99)), "mean_s": float(lat.mean()),
           "value": float(sum(work)) / makespan, "unit": UNIT, "makespan_s": makespan,
           "rounds": stats["rounds"], "peak_footprint_bytes": stats["peak_footprint_bytes"],
           "policy": list(policy) if policy else "library default"}
    if run_fifo:
        out["fifo_unbatched_measured"] = fifo_run(specs, wls, dev, arrivals)
    if fifo_rates:
        out["fifo_computed_from_rates"] = {k: fifo_latencies(arrivals, work, r)
                                           for k, r in fifo_rates.items() if r}
    return out


def insitu_leg(n_total: int = 10_000_000, n_chunk: int = 1_000_000, fp64_sample: int = 10_000):
    """In-situ scale: 1e7 macro-particles from the LWFA bunch generator streamed as
    10 calls of 1e6 into one time step, 1024 log omega x 32 x 32 directions
    (1.05e13 updates), CIC shape of 0.1 um, read out with CIC and TSC.  Reports
    the mixed path's rate and the accumulate kernel's roofline fraction; the
    plain FP64 kernel on a sample of the same step (fp64_sample particles of the
    first call, all bins: its work per update is uniform, so the rate carries
    over); and both readouts against the oracle on 32 sampled bins with all 1e7
    particles."""
    import numpy as np
    import torch

    import oracle
    from paper_1802_03972_gb300 import inputs, rad
    omega = inputs.omega_log(1e14, 1e20, 1024)
    dirs = inputs.dirs_grid(0.01, 32, 32)
    chunks = [inputs.BetatronBunch(n_chunk, seed=300 + i).step(0.0, 1e-16)
              for i in range(n_total // n_chunk)]
    dev = [[torch.from_numpy(a).cuda() for a in (st.r, st.beta, st.beta_dot, st.w)] for st in chunks]
    upd = n_total * omega.shape[0] * dirs.shape[0]
    ctx = rad.Context(omega, dirs, rad.FF_CIC, 0.1e-6)
    tile = ctx.tune(n_chunk)
    ctx.accumulate(*dev[0], 0.0, 1e-16)
    ctx.sync()
    ctx.reset()
    ctx.profile(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for d in dev:
        ctx.accumulate(*d, 0.0, 1e-16)
    e1.record()
    torch.cuda.synchronize()
    el = e0.elapsed_time(e1) / 1e3
    _, acc_ms, calls = ctx.profile_read()
    mhz = ctx.profile_clock()
    ctx.profile(False)
    sm = torch.cuda.get_device_properties(0).multi_processor_count
    peak = sm * MUFU_PER_CLK_SM * SM_MAX_MHZ * 1e6 / MUFU_PER_UPDATE
    achieved = upd / (acc_ms / 1e3)
    out = {"workload": "1e7 macro-particles (10 calls of 1e6), 1024 log omega 1e14-1e20 rad/s, "
                       "32x32 directions +-10 mrad, CIC 0.1 um; readouts CIC and TSC",
           "updates_per_step": upd, "value": upd / el, "unit": UNIT, "s_per_step": el,
           "tile": list(tile), "kernel_frac_of_mufu_roofline": achieved / peak,
           "sm_mhz_in_kernel": mhz}
    times = {}
    for name, ff in (("cic", None), ("tsc", (rad.FF_TSC, 0.1e-6))):
        ctx.spectrum(ff=ff)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        got = ctx.spectrum(ff=ff)
        b.record()
        torch.cuda.synchronize()
        times[name] = (got, a.elapsed_time(b))
    out["readout_ms"] = {k: v[1] for k, v in times.items()}
    # plain FP64 kernel on a sample of the step
    c64 = rad.Context(omega, dirs, rad.FF_CIC, 0.1e-6, prec=rad.PREC_FP64)
    def first(k):  # the first k particles of the first call, SoA [3][k] and [k]
        return ([x.reshape(3, n_chunk)[:, :k].contiguous().reshape(-1) for x in dev[0][:3]]
                + [dev[0][3][:k].contiguous()])

    c64.accumulate(*first(256), 0.0, 1e-16)  # warm-up
    c64.sync()
    sample = first(fp64_sample)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    c64.accumulate(*sample, 0.0, 1e-16)
    b.record()
    torch.cuda.synchronize()
    v64 = fp64_sample * omega.shape[0] * dirs.shape[0] / (a.elapsed_time(b) / 1e3)
    c64.close()
    out["fp64_plain"] = {"value": v64, "unit": UNIT, "mixed_over_fp64": (upd / el) / v64,
                         "sample": f"{fp64_sample} particles of the first call x all "
                                   f"{omega.shape[0] * dirs.shape[0]} bins, rate taken as "
                                   "the full step's (uniform work per update)"}
    # sampled bins against the oracle, both readouts
    rng = np.random.default_rng(4)
    bins = [(int(rng.integers(0, 1024)), int(rng.integers(0, 1024))) for _ in range(32)]
    bo, bd = oracle.grid_bins(omega, dirs, bins)
    acc = oracle.Accumulator(bo, bd, oracle.FF_CIC, 0.1e-6)
    t0 = time.perf_counter()
    for st in chunks:
        acc.accumulate(st.r, st.beta, st.beta_dot, st.w, st.t, st.dt)
    el_oracle = time.perf_counter() - t0
    out["oracle"] = {"value": len(bins) * n_total / el_oracle, "unit": UNIT,
                     "cores": oracle.num_threads(),
                     "sample": f"{len(bins)} sampled bins x all {n_total} particles of the step"}
    acc_out = {}
    for name, kind in (("cic", oracle.FF_CIC), ("tsc", oracle.FF_TSC)):
        ref = acc.spectra(kind, 0.1e-6)
        got = times[name][0]
        worst = 0.0
        for i, (d, o) in enumerate(bins):
            for k, g in zip(("coh", "inc", "tot"), got):
                m = float(np.abs(g[d]).max())
                r = float(ref[k][i])
                allowed = BIN_REL * r + 2.0 * BIN_AMP * math.sqrt(r * m) + BIN_AMP ** 2 * m
                if allowed > 0:
                    worst = max(worst, abs(float(g[d, o]) - r) / allowed)
        tot_rel = [abs(float(got[2][d, o]) - float(ref["tot"][i])) / float(ref["tot"][i])
                   for i, (d, o) in enumerate(bins) if ref["tot"][i] > 0]
        acc_out[name] = {"bin_excess": worst, "tot_bin_rel_max": max(tot_rel)}
    out["vs_oracle_32_sampled_bins"] = acc_out
    ctx.close()
    return out


def helix_leg():
    """The tiny helix workload (64 point particles, 1000 steps of 1e-17 s, 128 x 16
    bins): the mixed path and the plain FP64 kernel over all 1000 steps through
    the C ABI (device arrays resident), the oracle on the full grid on the host
    cores, and both GPU paths' errors against it."""
    import numpy as np
    import torch

    import oracle
    from paper_1802_03972_gb300 import inputs, rad
    wl = inputs.tiny_helix()
    steps = [wl.step(s) for s in range(wl.n_steps)]
    dev = [[torch.from_numpy(a).cuda() for a in (st.r, st.beta, st.beta_dot, st.w)] for st in steps]
    upd = wl.updates_per_step() * wl.n_steps
    out = {"workload": "64 point macro-particles on gamma = 50 helices, 1000 steps of 1e-17 s, "
                       "128 linear omega 1e15-1e18 rad/s x 16 directions 0-20 mrad",
           "updates": upd}
    spectra = {}
    for name, prec in (("mixed", rad.PREC_MIXED), ("fp64_plain", rad.PREC_FP64)):
        ctx = rad.Context(wl.omega, wl.dirs, wl.ff_kind, wl.ff_width, prec=prec)
        ctx.accumulate(*dev[0], steps[0].t, steps[0].dt)  # warm-up
        ctx.reset()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for d, st in zip(dev, steps):
            ctx.accumulate(*d, st.t, st.dt)
        e1.record()
        torch.cuda.synchronize()
        out[name] = {"value": upd / (e0.elapsed_time(e1) / 1e3), "unit": UNIT}
        spectra[name] = dict(zip(("coh", "inc", "tot"), ctx.spectrum()))
        ctx.close()
    bo, bd = oracle.grid_bins(wl.omega, wl.dirs)
    acc = oracle.Accumulator(bo, bd, wl.ff_kind, wl.ff_width)
    t0 = time.perf_counter()
    for st in steps:
        acc.accumulate(st.r, st.beta, st.beta_dot, st.w, st.t, st.dt)
    el = time.perf_counter() - t0
    out["oracle"] = {"value": upd / el, "unit": UNIT, "cores": oracle.num_threads(),
                     "sample": "the full grid, all steps"}
    shape = (wl.dirs.shape[0], wl.omega.shape[0])
    ref = {k: v.reshape(shape) for k, v in acc.spectra().items()}
    for name in ("mixed", "fp64_plain"):
        out[name]["vs_oracle"] = {k: error_stats(spectra[name][k], ref[k]) for k in ("tot", "coh")}
    return out


def horizon_leg(wl, tile, n_steps: int = 256, row: int = 200, stride: int = 4):
    """Accuracy over the workload's horizon: the timed tile for n_steps distinct
    steps of the headline workload, read out after 16, 64 and n_steps steps,
    against the oracle on one direction x every stride-th frequency."""
    import torch

    import oracle
    from paper_1802_03972_gb300 import rad
    n_om = wl.omega.shape[0]
    cols = list(range(0, n_om, stride))
    bo, bd = oracle.grid_bins(wl.omega, wl.dirs, [(row, o) for o in cols])
    acc = oracle.Accumulator(bo, bd, wl.ff_kind, wl.ff_width)
    ctx = rad.Context(wl.omega, wl.dirs, wl.ff_kind, wl.ff_width)
    ctx.set_tile(*tile)
    out = {"direction": row, "frequencies": f"every {stride}th of {n_om}", "readouts": {}}
    for s in range(n_steps):
        st = wl.step(s)
        ctx.accumulate(*[torch.from_numpy(a).cuda() for a in (st.r, st.beta, st.beta_dot, st.w)],
                       st.t, st.dt)
        acc.accumulate(st.r, st.beta, st.beta_dot, st.w, st.t, st.dt)
        if s + 1 in (16, 64, n_steps):
            got = dict(zip(("coh", "inc", "tot"), ctx.spectrum()))
            ref = acc.spectra()
            out["readouts"][str(s + 1)] = {k: error_stats(got[k][row][cols][None, :], ref[k][None, :])
                                          for k in ("tot", "coh", "inc")}
    ctx.close()
    return out


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    from paper_1802_03972_gb300 import inputs
    wl = inputs.lwfa_bunch(seed=2 + rank)
    if args.impl == "reference":
        if rank == 0:
            reference_arm(args, wl)
        return

    import numpy as np
    import torch

    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_1802_03972_gb300 import build, rad
    build.build()
    rad.load()
    dev = torch.device("cuda", local)

    # Resident inputs: a ring of distinct steps.
    ring = max(1, min(args.ring, args.steps + args.warmup))
    steps_host = [wl.step(s) for s in range(ring)]
    ring_dev = [[torch.from_numpy(a).to(dev) for a in (st.r, st.beta, st.beta_dot, st.w)]
                for st in steps_host]
    upd = wl.updates_per_step()
    if args.wide_only:
        tile = tuple(int(x) for x in args.tile.split(",")) if args.tile else (9, 512, 0)
        print(json.dumps({"wide_bunch": wide_leg(wl, tile, n_steps=args.steps)}), flush=True)
        return
    ctx = rad.Context(wl.omega, wl.dirs, wl.ff_kind, wl.ff_width)
    if args.tile:
        ctx.set_tile(*[int(x) for x in args.tile.split(",")])
        tile = ctx.get_tile()
    else:
        tile = ctx.tune(wl.n_particles) if not args.no_tune else ctx.get_tile()

    def run(k):
        st = steps_host[k % ring]
        ctx.accumulate(*ring_dev[k % ring], st.t + (k // ring) * ring * st.dt, st.dt)

    for k in range(args.warmup):
        run(k)
    ctx.sync()
    ctx.reset()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clk = Clocks(local)
    time.sleep(0.3)
    launches0 = rad.kernel_launch_count()
    ctx.profile(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for k in range(args.steps):
        run(k)
    e1.record()
    torch.cuda.synchronize()
    elapsed_ms = e0.elapsed_time(e1)
    clocks = clk.stop()
    launches = rad.kernel_launch_count() - launches0
    pre_ms, acc_ms, calls = ctx.profile_read()
    eff_mhz = ctx.profile_clock()
    ctx.profile(False)
    if dist:
        t = torch.tensor([elapsed_ms], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        elapsed_ms = float(t.item())
        dist.barrier()
    value = world * args.steps * upd / (elapsed_ms / 1e3)

    # N > 1: the ranks' particles are shards of one job (same grids and times,
    # each rank's own particles).  Its one exchange: rank 0 merges every rank's
    # state blob at readout (rad_state_export -> gather -> rad_state_merge).
    sharded = None
    if dist:
        from paper_1802_03972_gb300.multirank import merge_to_root
        dist.barrier()
        m0 = time.perf_counter()
        blob = ctx.state_export()
        merge_to_root(blob, ctx.state_merge)
        dist.barrier()
        sharded = {"ranks": world, "merge_s": time.perf_counter() - m0,
                   "state_bytes_per_rank": len(blob),
                   "pattern": "particles of one job sharded over the ranks; one state merge "
                              "on rank 0 at readout, outside the timed steps"}

    # Parity of the timed configuration (tile choice included) on two sampled
    # directions x all frequencies: the per-direction relative spectral error.
    rel_err = accuracy = None
    if rank == 0:
        import oracle
        oracle.build()
        chk = rad.Context(wl.omega, wl.dirs, wl.ff_kind, wl.ff_width)
        chk.set_tile(*ctx.get_tile())
        rows = [5, 200]
        n_om = wl.omega.shape[0]
        bins = [(d, o) for d in rows for o in range(n_om)]
        bo, bd = oracle.grid_bins(wl.omega, wl.dirs, bins)
        acc = oracle.Accumulator(bo, bd, wl.ff_kind, wl.ff_width)
        for k in range(2):
            st = steps_host[k]
            chk.accumulate(*ring_dev[k], st.t, st.dt)
            acc.accumulate(st.r, st.beta, st.beta_dot, st.w, st.t, st.dt)
        got = dict(zip(("coh", "inc", "tot"), chk.spectrum()))
        ref = {k: v.reshape(len(rows), n_om) for k, v in acc.spectra().items()}
        accuracy = {"vs_oracle": {"directions": rows, "steps": 2},
                    "gate": "row <= 1e-5 on tot, coh and inc"}
        for k in ("tot", "coh", "inc"):
            accuracy["vs_oracle"][k] = error_stats(got[k][rows], ref[k])
        rel_err = accuracy["vs_oracle"]["tot"]["row"]
        chk.close()

    # Roofline of the accumulate kernel (MUFU-bound: 2 sin/cos per update).
    sm = torch.cuda.get_device_properties(dev).multi_processor_count
    acc_s = acc_ms / max(calls, 1) / 1e3
    achieved = upd / acc_s if acc_s > 0 else None
    peak = sm * MUFU_PER_CLK_SM * SM_MAX_MHZ * 1e6 / MUFU_PER_UPDATE
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": UNIT,
            "frac": achieved / peak if achieved else None, "traffic": traffic_per_launch(upd, tile),
            "kernel": "accumulate_kernel variant %d (%s), omega tile %d, chunk %s" % (
                tile[0], VARIANT_NAMES.get(tile[0], "?"), tile[1],
                tile[2] or "auto"),
            "peak_basis": f"{sm} SMs x {MUFU_PER_CLK_SM:g} MUFU sin/cos per clk x {SM_MAX_MHZ:g} MHz "
                          f"(max SM clock) / {MUFU_PER_UPDATE:g} per update",
            "prepass_ms_per_step": pre_ms / max(calls, 1),
            "accumulate_ms_per_step": acc_ms / max(calls, 1)}
    if clocks.get("sm_mhz"):
        roof["frac_at_sampled_clock"] = achieved / (peak * clocks["sm_mhz"] / SM_MAX_MHZ)
    if eff_mhz > 0:
        # the SM clock the accumulate kernel actually ran at (its CTAs' cycle
        # counters over elapsed time), and the fraction of the peak at that clock
        roof["sm_mhz_in_kernel"] = eff_mhz
        roof["frac_at_kernel_clock"] = achieved / (peak * eff_mhz / SM_MAX_MHZ)

    # End to end through the C ABI with pinned host buffers: H2D of each step's
    # particles inside rad_accumulate, D2H of the spectra by rad_spectrum.
    e2e = None
    if not args.no_e2e:
        n_e2e = min(args.steps, 20)
        pinned = []
        for st in steps_host[:min(ring, 8)]:
            pinned.append([torch.from_numpy(a).pin_memory() for a in (st.r, st.beta, st.beta_dot, st.w)])
        # the spectra come back into pinned host buffers, as the particles go in
        outs = [torch.zeros((wl.dirs.shape[0], wl.omega.shape[0]), dtype=torch.float64).pin_memory()
                for _ in range(3)]
        ectx = rad.Context(wl.omega, wl.dirs, wl.ff_kind, wl.ff_width)
        if args.tile:
            ectx.set_tile(*tile)
        elif not args.no_tune:
            ectx.tune(wl.n_particles)  # the shape's tuned tile, from the tuner's cache
        ectx.accumulate(*pinned[0], steps_host[0].t, steps_host[0].dt)
        ectx.spectrum(out=outs)
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(n_e2e):
            st = steps_host[k % len(pinned)]
            ectx.accumulate(*pinned[k % len(pinned)], st.t, st.dt)
            ectx.spectrum(out=outs)
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        if dist:
            t = torch.tensor([el], device=dev, dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            el = float(t.item())
        e2e = {"value": world * n_e2e * upd / el, "unit": UNIT,
               "h2d_bytes_per_step": int(sum(a.numel() * 8 for a in pinned[0])),
               "d2h_bytes_per_step": int(sum(o.numel() * o.element_size() for o in outs)), "steps": n_e2e}
        ectx.close()

    # The plain FP64 GPU kernel on the same GPU (2 steps).
    fp64 = None
    if not args.no_fp64 and rank == 0:
        c64 = rad.Context(wl.omega, wl.dirs, wl.ff_kind, wl.ff_width, prec=rad.PREC_FP64)
        st = steps_host[0]
        c64.accumulate(*ring_dev[0], st.t, st.dt)
        c64.sync()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record()
        for k in range(2):
            st = steps_host[k + 1]
            c64.accumulate(*ring_dev[k + 1], st.t, st.dt)
        f1.record()
        torch.cuda.synchronize()
        v64 = 2 * upd / (f0.elapsed_time(f1) / 1e3)
        fp64 = {"value": v64, "unit": UNIT, "steps": 2, "mixed_over_fp64": value / world / v64}
        # the timed mixed configuration against the FP64 kernel on the full grid, same 3 steps
        cmx = rad.Context(wl.omega, wl.dirs, wl.ff_kind, wl.ff_width)
        cmx.set_tile(*ctx.get_tile())
        for k in range(3):
            st = steps_host[k]
            cmx.accumulate(*ring_dev[k], st.t, st.dt)
        gm = dict(zip(("coh", "inc", "tot"), cmx.spectrum()))
        g64 = dict(zip(("coh", "inc", "tot"), c64.spectrum()))
        fp64["mixed_vs_fp64_full_grid"] = {k: error_stats(gm[k], g64[k]) for k in ("tot", "coh", "inc")}
        cmx.close()
        c64.close()

    horizon = None
    if rank == 0 and not args.no_horizon:
        horizon = horizon_leg(wl, ctx.get_tile())

    cpu = None
    if not args.no_cpu and rank == 0 and world == 1:
        rate, cores, desc, _ = cpu_oracle_rate(wl, 64, 10.0)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc}

    modes = None
    if rank == 0 and not args.no_modes:
        modes = modes_leg(wl, ring_dev, steps_host, upd)
        modes["wide_bunch"] = wide_leg(wl, ctx.get_tile())
        modes["wide_bunch"]["over_headline"] = modes["wide_bunch"]["value"] / (value / world)

    insitu = None
    if rank == 0 and not args.no_insitu:
        insitu = insitu_leg()
    helix = None
    if rank == 0 and not args.no_helix:
        helix = helix_leg()

    batched = batched_small = None
    if not args.no_batch and rank == 0:
        batched = batch_leg(args.batch_rounds)
        from paper_1802_03972_gb300 import inputs as _inputs
        small = _inputs.job_mix(64, base_seed=4500, n_lo=1e3, n_hi=1e4, log2_omega=(6, 8),
                                log2_side=(2, 3))
        batched_small = batch_leg(max(args.batch_rounds, 10), specs=small,
                                  mix="64 small jobs: N log-uniform 1e3-1e4, 64-256 omega, "
                                      "16-64 directions")
    served = served_literal = None
    if not args.no_serve and rank == 0:
        single = batched["unbatched_value"] if batched else value / world
        fifo = {"fp64_plain": fp64["value"] if fp64 else None}
        pol = tuple(int(float(x)) for x in args.serve_policy.split(",")) if args.serve_policy else None
        lo, hi = (int(x) for x in args.serve_steps.split(","))
        served = serve_leg(args.serve_jobs, args.serve_load, args.serve_rate, steps_range=(lo, hi),
                           cap=single, fifo_rates=fifo, policy=pol,
                           run_fifo=not args.no_fifo_run)
        # the literal arrival rate of the serving workload: 200 jobs/s over a window of
        # 256 arrivals (steps per job scaled further so the backlog drains in seconds)
        served_literal = serve_leg(256, args.serve_load, 200.0, steps_range=(2, 8), seed=6,
                                   cap=single, fifo_rates={"mixed_single_job": single, **fifo},
                                   policy=pol)

    peaks = None
    if args.peaks and rank == 0:
        p = rad.probe_peaks()
        peaks = {"ffma_lanes_per_clk_sm": p[0], "ffma2_lanes_per_clk_sm": p[2],
                 "mufu_per_clk_sm": p[4], "dfma_per_clk_sm": p[6], "probe_mhz": p[5]}
        q = rad.probe_tensor()
        peaks["tensor"] = {"mma_sync_tf32_mac_per_clk_sm": q[0],
                           "tcgen05_tf32_clk_per_mma_n16_64_128_256": list(q[1:5]),
                           "tcgen05_f16_clk_per_mma_n16_256": list(q[5:7]), "probe_mhz": q[7]}
        lp = rad.probe_loop()
        peaks["update_loop_mufu_per_clk_sm"] = {
            "variant8": lp[0], "no_split": lp[2], "no_mma": lp[4], "neither": lp[6], "variant9": lp[8],
            "probe_mhz": [lp[i] for i in range(1, 10, 2)]}

    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
               "steps": args.steps, "warmup": args.warmup,
               "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": "f32", "data": "synthetic",
               "config": config(wl, {"parallelism": "1 GPU" if world == 1 else
                                     f"particles of one job sharded over {world} ranks "
                                     f"({wl.n_particles} per rank)"}),
               "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
               "clocks": clocks, "rel_err_sampled": rel_err, "accuracy": accuracy, "fp64_plain": fp64,
               "modes": modes, "batched": batched, "batched_small_jobs": batched_small,
               "insitu_scale": insitu, "tiny_helix": helix, "accuracy_horizon": horizon,
               "sharded": sharded,
               "serving": served,
               "serving_literal_rate": served_literal,
               "p50_s": served["p50_s"] if served else None,
               "p99_s": served["p99_s"] if served else None}
        if peaks:
            out["peaks"] = peaks
        print(json.dumps(out), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
