#!/usr/bin/env python
"""Benchmark of one SPH-with-boids step on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Workload (default): the large tank -- 2,097,152 fluid particles uniform in
the lower 40% of a 4x2x2 tank, settled for 200 steps, then 16,384 boids in 8
schools released; K timed steps.  A step is one call of sph_step: binning,
density, forces + integration, boid binning and rules (all in the library's
CUDA kernels).  Each timed step is bracketed by CUDA events on the step's
stream; L2 is flushed (a 256 MiB write) between timed steps, outside the
events.  ``value`` = fluid particles x steps / summed step time (max over
ranks; under torchrun every rank runs its own replica: weak scaling).

Also reported: per-pass times (library event hook), the roofline of the
dominant pass, the CPU oracle on a bounded sample, an end-to-end figure
through host buffers, kernel launches and SM clocks.

``--impl reference`` times the CPU oracle (the reference program of this
method) on the same workload: each step is the full oracle step on a
bounded spatial sample of the tank.
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
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2311_15088_gb300 import scenes  # noqa: E402

METRIC = "particle-steps/sec at 2M particles (HBM roofline %)"
UNIT = "particle-steps/s"
SETTLE = 200

# FP32 peak of the ALU-bound passes: SMs x 128 FP32 lanes x 2 flops (FMA) x
# the maximum SM clock.  Set by _set_fp32_peak from the device's SM count and
# the measured peaks' maximum clock once the device is known; the nominal
# GB300 figure (152 SMs, 2070 MHz) until then.
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12
FP32_PEAK_SOURCE = "derived: 152 SMs x 128 FP32 lanes x 2 x 2070 MHz"


def _set_fp32_peak(dev):
    global FP32_PEAK_TFLOPS, FP32_PEAK_SOURCE
    import torch

    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = 2070.0
    try:
        mhz = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))).get("sm_max_mhz", mhz))
    except (OSError, ValueError):
        pass
    FP32_PEAK_TFLOPS = sms * 128 * 2 * mhz * 1e6 / 1e12
    FP32_PEAK_SOURCE = f"derived: {sms} SMs x 128 FP32 lanes x 2 x {mhz:.0f} MHz"
# Algorithmic work per particle-step, as the method defines it: each pass
# tests the candidates of the 27-cell stencil of cell size h, C = 27 n h^3
# per particle (n the number density), i.e. C = N * 27 / (4 pi / 3) with N
# = (4 pi / 3) n h^3 the neighbour count; a candidate test is 9 flops (3 sub,
# 3 mul / fma, compare), a density pair 5 flops, a force pair 35 flops.
# "executed" counts what the kernels actually do (read back from the
# library): the density pass tests the candidates of its pruned walk once
# for both passes and stores the hits as segments; the force pass evaluates
# the stored pairs (the particle itself included, then discarded) and tests
# candidates again only for the particles whose segments overflowed.
FLOP_CAND, FLOP_DENS_PAIR, FLOP_FORCE_PAIR = 9, 5, 35
STENCIL_CAND_PER_NBR = 27.0 / (4.0 * math.pi / 3.0)
SEG_CAP = 128  # hit segments stored per particle
# Compulsory bytes per particle of each pass (the method's minimum, float4
# pos/vel, float rho): binning key + rank (scatter 12) and the gather of
# pos, vel (sort 60), density pos in / rho out (20), forces pos, vel, rho in,
# pos, vel, key out (72).  The kernels move more: the density pass writes
# the hit segments and pair records the force pass reads (ncu traffic below).
BYTES = {"scatter": 12, "sort": 60, "density": 20, "forces": 72}
BYTES_PER_CELL_SCAN = 12

# DRAM traffic per launch of the force and density passes from one ncu
# capture of the bench's workload, and the sha256 of the kernel sources
# (sph_physics.cu, sph_internal.cuh) it was taken on; null once they moved.
# Capture: the launch list (gpu__time_duration, dram__bytes_read/write, one
# pass) of `bench.py --steps 20 --warmup 3 --no-cpu-baseline --e2e-steps 2
# --no-batch --no-surrogate --no-surface`, mean over the 21 launches of the
# timed steps after 200 settling steps (k_forces: the fluid launches).
KERNEL_TRAFFIC = {
    "k_forces": {"bytes": 720.4e6, "read": 643.0e6, "write": 77.4e6,
                 "source_sha256": "6b796b8c825557b856e8bbf3bfed9d904664eaa34e59dceed01518a5c17eb9c8"},
    "k_density": {"bytes": 864.2e6, "read": 289.4e6, "write": 574.8e6,
                  "source_sha256": "6b796b8c825557b856e8bbf3bfed9d904664eaa34e59dceed01518a5c17eb9c8"},
}


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--workload", choices=("large", "column", "small"), default="large")
    ap.add_argument("--e2e-steps", type=int, default=None,
                    help="steps of the end-to-end leg (default: the K timed steps, from the same state)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="approximate CPU time of the oracle baseline sample")
    ap.add_argument("--reference-budget", type=float, default=150.0,
                    help="seconds the reference arm may spend on its K + W sample steps")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batch-steps", type=int, default=30, help="timed steps of the batched-scenes leg")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-surrogate", action="store_true")
    ap.add_argument("--no-surface", action="store_true", help="skip the voxel density + marching cubes leg")
    ap.add_argument("--neighbor-lists", action="store_true",
                    help="build neighbour lists every step (pair buffer of 3x the pairs after warm-up) "
                         "and read them in the force pass instead of testing candidates")
    ap.add_argument("--mlp-throughput", action="store_true",
                    help="only time the surrogate network's forward pass on 65,536 queries (features of "
                         "the 262,144-particle column's 1,024 boids, tiled), untrained weights")
    ap.add_argument("--cell-x", type=float, default=None,
                    help="particle-grid cell size along x over h for the main leg (default: the workload's)")
    ap.add_argument("--settle", type=int, default=None,
                    help="settling steps of the large tank before the boids are released (default 200)")
    return ap.parse_args()


def _workload(name):
    if name == "large":
        sc = scenes.large_tank()
        desc = ("large tank: 2,097,152 fluid particles uniform in the lower 40% of a 4x2x2 tank, "
                f"settled {SETTLE} steps, then 16,384 boids in 8 schools")
        return sc, desc, SETTLE
    if name == "column":
        sc = scenes.dam_break_column()
        return sc, "dam-break column: 262,144 particles (64^3 lattice) in a 2x1x1 tank, 1,024 boids", 0
    sc = scenes.dam_break_small()
    return sc, "dam-break: 4,096 particles (16^3 lattice) in the unit box, 16 boids", 0


def _params(sc):
    p = dict(sc["params"])
    if p.get("mass") is None:
        from paper_2311_15088_gb300 import sph

        p["mass"] = sph.sph_lattice_mass(p, sc["lattice_spacing"])
    return p


def _max_over_ranks(t: float, world: int, dev) -> float:
    """The slowest rank's timed seconds (every rank gets it)."""
    if world <= 1:
        return t
    import torch

    tt = torch.tensor([t], dtype=torch.float64, device=dev)
    torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
    return float(tt.item())


def _job_value(n_fluid: int, steps: int, world: int, seconds: float) -> float:
    """Whole-job particle-steps/s: every rank steps its own replica."""
    return n_fluid * steps * world / seconds


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons (read only)."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            time.sleep(1.0)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for nm, val in zip(names, f[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------- work counts

def _work_snapshot(s):
    """Candidates tested, neighbour pairs, hit segments stored and the
    candidates of the particles whose segments overflowed (tested again by
    the force pass), for the step last run."""
    nc = s.field("ncand").cpu().numpy().astype(np.int64)
    nbr = s.field("nbr_count").cpu().numpy()
    nseg = s.field("nseg").cpu().numpy().astype(np.int64)
    from paper_2311_15088_gb300.sph import STATS
    st = s.stats().cpu().numpy()[0]
    over = nseg > SEG_CAP
    return {"candidates": int(nc.sum()), "pairs": int(nbr.astype(np.int64).sum()),
            "segments": int(nseg[~over].sum()), "overflow_particles": int(over.sum()),
            "overflow_candidates": int(nc[over].sum()),
            "nbr_mean": float(nbr.mean()), "nbr_max": int(nbr.max()),
            "stats": {k: float(v) for k, v in zip(STATS, st)}}


def _source_sha(*paths):
    """sha256 over the concatenated bytes of the kernel sources."""
    h = hashlib.sha256()
    for path in paths:
        h.update(open(path, "rb").read())
    return h.hexdigest()


# ------------------------------------------------------- neighbour search

def _neighbor_search(s, dev):
    """Neighbour counts of the current state by the exact walk and by the
    fixed-capacity hash grid (buckets of twice the most crowded cell of the
    previous binning, and of 16 entries): times (binning included, CUDA
    events) and the fraction of neighbour pairs the 16-entry buckets lose."""
    import torch

    def timed(fn):
        fn()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        out = fn()
        e1.record()
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1), out

    s.step(1)  # (the end-to-end leg's host downloads staged through the step's scratch)
    occupancy = int(torch.diff(s.field("cell_start").to(torch.int64)).max().item())  # of that step's binning
    ms_walk, (exact, _, _) = timed(lambda: s.neighbors(lists=False))
    ms_full, (full, dropped_full) = timed(lambda: s.bucket_neighbors(2 * occupancy))
    ms_16, (c16, dropped) = timed(lambda: s.bucket_neighbors(16))
    pairs = float(exact.to(torch.float64).sum().item())
    return {"walk_ms": ms_walk, "bucket_ms": ms_full, "bucket_capacity": 2 * occupancy,
            "bucket_dropped_particles": int(dropped_full.item()),
            "bucket_equals_walk": bool(torch.equal(full, exact)),
            "bucket16_ms": ms_16, "bucket16_dropped_particles": int(dropped.item()),
            "bucket16_lost_pair_fraction": 1.0 - float(c16.to(torch.float64).sum().item()) / max(pairs, 1.0)}


# ------------------------------------------------------------ surface

def _surface(s, dev, p, warmup=3, reps=10):
    """Surface reconstruction of the current state (the paper's third stage):
    voxel density on the corner grid over the box at spacing h/2 (R = h,
    particle radius h/4), then marching cubes into a device triangle buffer;
    CUDA-event times (mean of ``reps`` after ``warmup``), the voxel pass's
    roofline against the FP32 ALU peak (9 flops per candidate tested, 20 per
    neighbour) and the marching-cubes pass's against the HBM peak (corner
    values read once, triangles written: compulsory bytes)."""
    import torch

    from paper_2311_15088_gb300 import sph

    h = float(np.float32(p["h"]))
    sp, R, r = float(np.float32(h * 0.5)), float(np.float32(h)), float(np.float32(h * 0.25))
    origin, dims = sph.sph_voxel_grid(p, sp, R)
    n = dims[0] * dims[1] * dims[2]
    phi = torch.empty(n, dtype=torch.float32, device=dev)
    cnt = torch.empty(n, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev).cuda_stream
    ncubes = (dims[0] - 1) * (dims[1] - 1) * (dims[2] - 1)
    ws_bytes = sph.sph_mc_workspace_size(dims)
    ws = torch.empty(ws_bytes + 256, dtype=torch.uint8, device=dev)
    ws_ptr = (ws.data_ptr() + 255) & ~255
    cap = 4 << 20
    tris = torch.empty((cap, 9), dtype=torch.float32, device=dev)
    ntri = torch.zeros(1, dtype=torch.int32, device=dev)

    def voxel():
        sph.sph_voxel_density(s.handle, origin, dims, sp, R, r, phi.data_ptr(), cnt.data_ptr(), stream)

    def mc():
        sph.sph_marching_cubes(phi.data_ptr(), dims, origin, sp, 0.0, ws_ptr, ws_bytes, tris.data_ptr(), cap,
                               ntri.data_ptr(), stream)

    def timed(fn):
        for _ in range(warmup):
            fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / reps

    ms_voxel = timed(voxel)  # includes the state's binning
    ms_mc = timed(mc)
    total = int(ntri.item())
    nbrs = float(cnt.to(torch.float64).sum().item())
    occupied = int((cnt > 0).sum().item())
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    flops = FLOP_CAND * STENCIL_CAND_PER_NBR * nbrs + 20 * nbrs
    mc_bytes = 4 * n + 36 * min(total, cap)
    return {"workload": "voxel density + marching cubes of the tank after the timed steps",
            "spacing": sp, "radius": R, "particle_radius": r, "corners": n, "cubes": ncubes,
            "corners_with_neighbours": occupied, "mean_neighbours_per_occupied_corner": nbrs / max(occupied, 1),
            "triangles": total, "voxel_ms": ms_voxel, "mc_ms": ms_mc,
            "corners_per_s": n / (ms_voxel * 1e-3), "triangles_per_s": total / (ms_mc * 1e-3),
            "voxel_roofline": {"bound": "alu", "achieved": flops / (ms_voxel * 1e-3) / 1e12, "peak": FP32_PEAK_TFLOPS,
                               "unit": "TFLOP/s", "frac": flops / (ms_voxel * 1e-3) / 1e12 / FP32_PEAK_TFLOPS,
                               "definition": "27-cell stencil at cell size R: 9 flops x 27/(4pi/3) x neighbours "
                                             "+ 20 x neighbours; time includes the binning"},
            "mc_roofline": {"bound": "hbm", "achieved": mc_bytes / (ms_mc * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s",
                            "frac": mc_bytes / (ms_mc * 1e-3) / 1e9 / hbm,
                            "definition": "4 B per corner read + 36 B per triangle written"}}


# --------------------------------------------------------------- CPU oracle

def _cpu_model() -> str:
    """The host CPU's name from /proc/cpuinfo (x86: model name; Arm: the
    implementer and part numbers), else the machine type."""
    import platform

    try:
        info = open("/proc/cpuinfo").read()
    except OSError:
        return platform.machine()
    for key in ("model name", "Model"):
        for line in info.splitlines():
            if line.startswith(key):
                return line.split(":", 1)[1].strip()
    impl = [ln.split(":", 1)[1].strip() for ln in info.splitlines() if ln.startswith("CPU implementer")]
    part = [ln.split(":", 1)[1].strip() for ln in info.splitlines() if ln.startswith("CPU part")]
    if impl and part:
        return f"{platform.machine()} implementer {impl[0]} part {part[0]}"
    return platform.machine()


def _slab(fp, fv, bp, bv, lo, hi):
    m = (fp[:, 0] >= lo) & (fp[:, 0] < hi)
    mb = (bp[:, 0] >= lo) & (bp[:, 0] < hi)
    return fp[m], fv[m], bp[mb], bv[mb]


def _oracle_rate(p, fp, fv, bp, bv, step_seconds, min_seconds=0.0, steps=None):
    """Full oracle steps on a centred x-slab of the state.  The slab is grown
    until one step takes about ``step_seconds``; then ``steps`` steps (or as
    many as fill ``min_seconds``) are timed.  Returns (particle-steps/s,
    threads, description, steps, particles, seconds)."""
    import oracle

    oracle.build()
    x0, x1 = float(p["box_min"][0]), float(p["box_max"][0])
    full = x1 - x0
    w = full * min(1.0, 20000.0 / max(len(fp), 1))
    for _ in range(8):
        lo = x0 + 0.5 * (full - w)
        sample = _slab(fp, fv, bp, bv, lo, lo + w)
        t = time.perf_counter()
        oracle.step(p, *sample)
        t = time.perf_counter() - t
        if t >= 0.6 * step_seconds or w >= full:
            break
        w = min(full, w * min(4.0, step_seconds / max(t, 1e-6)))
    n_steps, done, t0 = 0, 0, time.perf_counter()
    while True:
        oracle.step(p, *sample)
        n_steps += 1
        done += len(sample[0])
        el = time.perf_counter() - t0
        if (steps is not None and n_steps >= steps) or (steps is None and el >= min_seconds):
            break
    desc = (f"full oracle step on the x-slab [{lo:.3f}, {lo + w:.3f}) of the tank: {len(sample[0])} fluid "
            f"particles and {len(sample[2])} boids, {n_steps} step(s)")
    return done / el, oracle.num_threads(), desc, n_steps, len(sample[0]), el


# ------------------------------------------------------------- batched

# Cell shapes the batched leg tries (cell size over h along y and z, along
# x), each with the autotuner; the fastest is kept.
CELL_SHAPES = ((0.5, 0.5), (1.0, 1.0), (1.0, 0.5), (1.0, 0.34))


def run_batched(a, dev, flush):
    """256 independent tanks in one handle (every pass one launch over all
    scenes, the step replayed from a CUDA graph, launch shape autotuned)
    against a loop that replays each scene's own captured step with the same
    kernels.  The cell size is tuned too, over h/2 and h (it changes the
    float32 summation order, not the results beyond rounding: parity is
    tested at both); the loop uses the chosen one.  Under torchrun the
    scenes are split across the ranks (greedy bin-pack by particle count,
    paper_2311_15088_gb300.shard): each rank steps its share, the time is
    the slowest rank's and scenes/s counts all 256 (strong scaling of this
    leg).  Returns the "batched" object of the bench line."""
    import torch

    from paper_2311_15088_gb300 import shard, sph, tune
    from paper_2311_15088_gb300.sph import Scene

    world, rank, _ = _dist()
    all_scs = scenes.batched_tanks()
    for sc in all_scs:
        sc["params"] = _params(sc)
    S = len(all_scs)
    weights = [shard.scene_weight(sc) for sc in all_scs]
    parts = shard.assign(weights, world)
    scs = [all_scs[k] for k in parts[rank]]
    nf = [len(sc["fluid_pos"]) for sc in scs]
    nb = [len(sc["boid_pos"]) for sc in scs]
    nf_all = sum(len(sc["fluid_pos"]) for sc in all_scs)
    cat = lambda key: np.concatenate([sc[key] for sc in scs])
    stream = torch.cuda.Stream(dev)

    def with_cell(frac, frac_x):
        out = []
        for sc in scs:
            q = dict(sc["params"])
            q["cell_size"] = float(np.float32(np.float32(q["h"]) * np.float32(frac)))
            q["cell_size_x"] = float(np.float32(np.float32(q["h"]) * np.float32(frac_x)))
            out.append(q)
        return out

    def timed_steps(fn, n):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
        torch.cuda.synchronize(dev)
        for e0, e1 in ev:
            flush.zero_()
            e0.record()
            fn()
            e1.record()
        torch.cuda.synchronize(dev)
        return sum(e0.elapsed_time(e1) for e0, e1 in ev) / 1e3

    per_cell = {}
    with torch.cuda.stream(stream):
        for frac in CELL_SHAPES:
            ps = with_cell(*frac)
            b = Scene(ps, nf, nb, device=dev)
            b.set_state(cat("fluid_pos"), cat("fluid_vel"), cat("boid_pos"), cat("boid_vel"))
            best = tune.autotune(b, steps=3, cache=None)
            for _ in range(a.warmup):
                b.graph_step(1)
            l0 = b.launches
            t = timed_steps(lambda: b.graph_step(1), a.batch_steps)
            launches = b.launches - l0
            work = _work_snapshot(b)
            per_cell[frac] = {"t": _max_over_ranks(t, world, dev), "launches": launches, "tuning": best,
                              "params": ps, "work": work, "ncells": b.ncells}
            del b
        frac = min(per_cell, key=lambda f: per_cell[f]["t"])
        chosen = per_cell[frac]
        t_batch, launches, best = chosen["t"], chosen["launches"], chosen["tuning"]
        # the same scenes, one handle each, each replaying its own captured step
        loop = []
        for sc, q in zip(scs, chosen["params"]):
            s1 = Scene(q, len(sc["fluid_pos"]), len(sc["boid_pos"]), device=dev)
            s1.set_state(sc["fluid_pos"], sc["fluid_vel"], sc["boid_pos"], sc["boid_vel"])
            tune.apply(s1, best)
            loop.append(s1)
        for _ in range(max(a.warmup, 2)):
            for s1 in loop:
                s1.graph_step(1)
        n_loop = max(3, a.batch_steps // 3)

        def loop_step():
            for s1 in loop:
                sph.sph_graph_step(s1.handle, 1, stream.cuda_stream)

        t_loop = _max_over_ranks(timed_steps(loop_step, n_loop), world, dev)
        del loop
    cpu = None
    if not a.no_cpu_baseline and world == 1:
        # the oracle, as it stands, one step of every 16th scene (its cell size)
        import oracle

        oracle.build()
        picked = list(range(0, S, 16))
        t0 = time.perf_counter()
        for i in picked:
            sc = all_scs[i]
            oracle.step(chosen["params"][i], sc["fluid_pos"], sc["fluid_vel"], sc["boid_pos"], sc["boid_vel"])
        el = time.perf_counter() - t0
        nf_p = sum(len(all_scs[i]["fluid_pos"]) for i in picked)
        cpu = {"value": len(picked) / el, "unit": "scenes/s", "cores": oracle.num_threads(), "kind": "oracle",
               "particle_steps_per_s": nf_p / el,
               "sample": f"one oracle step of each of {len(picked)} scenes (every 16th), {nf_p} fluid particles"}
    # rooflines of this rank's batched step (its share of the scenes)
    ms = 1e3 * t_batch / a.batch_steps
    w = chosen["work"]
    n_all = sum(nf) + sum(nb)
    stencil = STENCIL_CAND_PER_NBR * w["pairs"]
    flops = 2 * FLOP_CAND * stencil + FLOP_DENS_PAIR * (w["pairs"] + n_all) + FLOP_FORCE_PAIR * w["pairs"]
    step_bytes = n_all * sum(BYTES.values()) + chosen["ncells"] * BYTES_PER_CELL_SCAN
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    return {
        "cpu_baseline": cpu,
        "workload": f"{S} unit-box dam-breaks, particles log-uniform in [2048, 65536], boids uniform in [8, 256]",
        "scenes": S, "particles": int(nf_all), "boids": int(sum(len(sc["boid_pos"]) for sc in all_scs)),
        "steps": a.batch_steps, "ranks": world, "scaling": "strong" if world > 1 else None,
        "scenes_per_rank": [len(p) for p in parts], "load_imbalance": shard.imbalance(weights, parts),
        "scenes_per_s": S * a.batch_steps / t_batch, "ms_per_step": 1e3 * t_batch / a.batch_steps,
        "particle_steps_per_s": nf_all * a.batch_steps / t_batch, "gpu_launches": launches,
        "loop_scenes_per_s": S * n_loop / t_loop, "loop_ms_per_step": 1e3 * t_loop / n_loop,
        "speedup_vs_loop": (S * a.batch_steps / t_batch) / (S * n_loop / t_loop),
        "loop": "each scene's own handle replaying its captured step (sph_graph_step), same kernels",
        "cell_size_over_h": frac[0], "cell_size_x_over_h": frac[1],
        "ms_per_step_by_cell_size": {f"{f[0]}/{f[1]}": 1e3 * v["t"] / a.batch_steps for f, v in per_cell.items()},
        "tuning": {k: best[k] for k in ("block", "use_segments", "ppt", "pipe_tile", "pipe_block", "ms_per_step")},
        "roofline": {
            "alu": {"achieved": flops / (ms * 1e-3) / 1e12, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "frac": flops / (ms * 1e-3) / 1e12 / FP32_PEAK_TFLOPS,
                    "definition": "both neighbour passes' algorithmic flops (27-cell stencil at h) over the whole "
                                  "step's time, this rank's scenes"},
            "hbm": {"achieved": step_bytes / (ms * 1e-3) / 1e9, "peak": hbm_peak, "unit": "GB/s",
                    "frac": step_bytes / (ms * 1e-3) / 1e9 / hbm_peak,
                    "definition": "compulsory bytes per particle-step (binning 72, density 20, forces 72) + 12 B "
                                  "per cell, over the whole step's time; the small scenes stay in L2"},
            "neighbours_mean": w["nbr_mean"]},
        "mode": "CUDA graph replay of one step; L2 flushed between timed steps",
    }


# ----------------------------------------------------------- surrogate

HEAD_ONLY = "surrogate_fallback_head_only"


def _time_modes(s, modes, n_states, warmup, bounds=None):
    """Per mode: summed ms of the boid-force call over n_states states (one
    step between states), the forces and the fallback flags.  Every mode is
    replayed from its captured graph (sph_graph_boid_forces, on the current
    stream, which must not be the default one), except the mode named
    HEAD_ONLY, the fallback with the input-range check off: switching the
    range drops the captured calls, so it runs plain calls, in a second pass
    over the same states (the state is restored from a snapshot)."""
    import torch

    graphed = {k: v for k, v in modes.items() if k != HEAD_ONLY}
    ms = {k: 0.0 for k in modes}
    got = {k: [] for k in modes}
    fall = {k: [] for k in modes if k.startswith("surrogate_fallback")}
    snapshot = [t.clone() for t in s.get_state()]

    def run(which, call):
        for _ in range(max(warmup, 2)):  # the plain first call, then the capture
            for name, mode in which.items():
                call(mode)
        for _ in range(n_states):
            for name, mode in which.items():
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                f = call(mode)
                e1.record()
                torch.cuda.synchronize()
                ms[name] += e0.elapsed_time(e1)
                got[name].append(f[:, :3].clone())
                if name in fall:
                    fall[name].append(f[:, 3].clone())
            s.step(1)

    run(graphed, s.graph_boid_forces)
    if HEAD_ONLY in modes:
        s.set_state(*snapshot)
        s.set_surrogate_bounds(None)
        run({HEAD_ONLY: modes[HEAD_ONLY]}, s.boid_forces)
        s.set_surrogate_bounds(bounds)
    return ms, got, fall


def _mode_report(surrogate, ms, got, fall, q, n_states):
    import torch

    F = torch.cat(got["exact_local"])
    out = {}
    for name in ms:
        med, p90 = surrogate.per_query_error(torch.cat(got[name]), F)
        out[name] = {"qps": q / (ms[name] / 1e3), "ms_per_state": ms[name] / n_states,
                     "aggregate_error": surrogate.aggregate_error(torch.cat(got[name]), F),
                     "per_query_error_median": med, "per_query_error_p90": p90}
    for name, fl in fall.items():
        out[name]["fallback_fraction"] = float(torch.cat(fl).mean().item())
    out["exact_local_equals_exact_full"] = bool(torch.equal(F, torch.cat(got["exact_full"])))
    out["speedup_surrogate_vs_exact_full"] = out["surrogate"]["qps"] / out["exact_full"]["qps"]
    out["speedup_at_5pct_vs_exact_full"] = out["surrogate_fallback"]["qps"] / out["exact_full"]["qps"]
    # the fastest mode whose measured aggregate error is within 5 %
    ok = [n for n in ms if out[n]["aggregate_error"] <= 0.05]
    best = max(ok, key=lambda n: out[n]["qps"])
    out["fastest_within_5pct"] = {"mode": best, "qps": out[best]["qps"],
                                  "aggregate_error": out[best]["aggregate_error"],
                                  "speedup_vs_exact_full": out[best]["qps"] / out["exact_full"]["qps"]}
    return out


def _features_roofline(s, dev, reps=20):
    """The surrogate's stencil features (the feature grid and k_features,
    timed together by the library's event hook): the compulsory bytes are
    every particle's position and every fluid particle's velocity read once
    by the grid pass (16 B each), the integer grid of h-cells zeroed and
    written once (16 B a cell) and one 544-byte feature row per boid; the
    gathers of a boid's 64 cells and h-neighbours hit L2.  Against the
    measured HBM peak."""
    import numpy as np
    import torch

    from paper_2311_15088_gb300 import sph

    sph.sph_profile_enable(s.handle, 4 * reps + 8)
    for _ in range(reps):
        s.features()
    torch.cuda.synchronize(dev)
    prof = sph.sph_profile_read(s.handle)
    sph.sph_profile_enable(s.handle, 0)
    ms, cnt = prof["features"]
    ms = ms / max(cnt, 1)
    p = s.params
    inv_h = np.float32(1.0) / np.float32(p["h"])
    ext = np.asarray(p["box_max"], np.float32) - np.asarray(p["box_min"], np.float32)
    fdim = np.floor(ext * inv_h).astype(np.int64) + 1 + 4  # two cells of margin per side
    ncells = int(np.prod(fdim))
    n_all = s.n_fluid + s.n_boid
    total = 16 * n_all + 16 * s.n_fluid + 16 * ncells + 544 * s.n_boid
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    gbs = total / (ms * 1e-3) / 1e9
    return {"kernel": "k_feature_grid + k_features", "ms_per_launch": ms, "boids": s.n_boid,
            "feature_cells": ncells, "bytes_per_launch": total,
            "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm, "bound": "hbm",
            "definition": "16 B position of every particle + 16 B velocity of every fluid particle + "
                          "16 B per feature cell + the 544-byte row of every boid"}


def _network_roofline(s, mlp, reps=50):
    """The trained network alone (the fused tcgen05 forward) on 65,536 rows:
    the state's 1,024 feature rows tiled 64 times; BF16 dense flops per
    launch over its CUDA-event time, against the measured BF16 peak."""
    import torch

    X = s.features().repeat(64, 1).contiguous()
    for _ in range(3):
        mlp.forward(X)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        mlp.forward(X)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    flops = 2.0 * X.shape[0] * (272 * 256 + 256 * 256 * 2 + 256 * 16)
    peak = None
    try:
        peak = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["bf16_tflops"])
    except (OSError, ValueError, KeyError):
        pass
    ach = flops / (ms * 1e-3) / 1e12
    return {"bound": "tensor", "kernel": "k_mlp_fused (4 layers, 65,536 rows)", "achieved": ach, "peak": peak,
            "unit": "TFLOP/s", "frac": ach / peak if peak else None, "ms_per_launch": ms,
            "queries_per_s": X.shape[0] / (ms * 1e-3), "flops_per_launch": flops,
            "peak_source": "measured (bf16 burst)" if peak else None}


def _oracle_surrogate(p, sc):
    """The oracle, as it stands, on the surrogate's work: stencil features of
    64 boids of the evaluation column state, the float64 network over
    65,536 rows (random rows of the feature width: the cost does not depend
    on the values), and one full oracle step of the state (which computes
    every boid's exact F_b)."""
    import oracle
    from oracle import features, mlp as omlp

    oracle.build()
    nb = 64
    t0 = time.perf_counter()
    features.stencil_features(p, sc["fluid_pos"], sc["fluid_vel"], sc["boid_pos"][:nb], sc["boid_vel"][:nb])
    t_feat = (time.perf_counter() - t0) / nb
    x = np.random.default_rng(0).normal(size=(65536, omlp.D_IN))
    params = omlp.init_params(0)
    t0 = time.perf_counter()
    omlp.forward(params, x)
    t_mlp = (time.perf_counter() - t0) / len(x)
    t0 = time.perf_counter()
    oracle.step(p, sc["fluid_pos"], sc["fluid_vel"], sc["boid_pos"], sc["boid_vel"])
    t_step = time.perf_counter() - t0
    return {"value": 1.0 / (t_feat + t_mlp), "unit": "queries/s", "kind": "oracle", "cores": oracle.num_threads(),
            "features_qps": 1.0 / t_feat, "network_fp64_qps": 1.0 / t_mlp,
            "exact_qps": len(sc["boid_pos"]) / t_step,
            "sample": f"features of {nb} boids; the float64 network on 65,536 rows; one full oracle step of the "
                      f"{len(sc['fluid_pos'])}-particle state with its {len(sc['boid_pos'])} boids (exact F_b)"}


def run_surrogate(a, dev, big=None):
    """Boid-force queries: the surrogate (features + tensor-core MLP), the
    surrogate with its exact fallback at the calibrated 5 % aggregate error,
    and the exact force computed only where it is needed, on 65,536 queries
    (64 states x 1,024 boids of held-out 262,144-particle column runs), and
    on the settled large tank ``big`` (4 states x 16,384 boids, a shift from
    the training distribution).  The network is trained first (untimed) on
    48 runs x 64 steps of the column with other seeds (40 epochs).  Each per-state time
    includes the state's binning, which every mode needs."""
    import torch

    from paper_2311_15088_gb300 import surrogate
    from paper_2311_15088_gb300.sph import (SPH_BOID_EXACT, SPH_BOID_EXACT_LOCAL, SPH_BOID_SURROGATE,
                                            SPH_BOID_SURROGATE_FALLBACK, Scene)

    mk = lambda sd: scenes.dam_break_column(seed_offset=100 + sd)
    # 48 training runs (3.1M pairs), 2 calibration runs, the evaluation run (40) held out
    train_runs = list(range(16)) + list(range(18, 40)) + list(range(41, 51))
    mlp, info = surrogate.build_and_train(mk, train_runs, [16, 17], steps=64, epochs=40)
    sc = mk(40)
    p = _params(sc)
    modes = {"exact_full": SPH_BOID_EXACT, "exact_local": SPH_BOID_EXACT_LOCAL, "surrogate": SPH_BOID_SURROGATE,
             "surrogate_fallback": SPH_BOID_SURROGATE_FALLBACK, HEAD_ONLY: SPH_BOID_SURROGATE_FALLBACK}
    n_states = 64
    stream = torch.cuda.Stream(dev)
    torch.cuda.synchronize(dev)
    with torch.cuda.stream(stream):
        s = Scene(p, len(sc["fluid_pos"]), len(sc["boid_pos"]), device=dev)
        s.set_state(sc["fluid_pos"], sc["fluid_vel"], sc["boid_pos"], sc["boid_vel"])
        s.set_surrogate(mlp, info["f_scale"], info["threshold"], mlp.bounds)
        ms, got, fall = _time_modes(s, modes, n_states, a.warmup, mlp.bounds)
        feat = _features_roofline(s, dev)
    out = {"workload": "65,536 boid-force queries: 64 states x 1,024 boids of a 262,144-particle column run",
           "training": info, "queries": n_states * s.n_boid,
           "mode": "each mode replayed from its captured graph (sph_graph_boid_forces)",
           "features_roofline": feat}
    out.update(_mode_report(surrogate, ms, got, fall, n_states * s.n_boid, n_states))
    out["network_roofline"] = _network_roofline(s, mlp)
    if not a.no_cpu_baseline:
        out["cpu_baseline"] = _oracle_surrogate(p, sc)
    if big is not None:
        # distribution shift: the settled 2M-particle tank and its 16,384 boids
        torch.cuda.synchronize(dev)
        with torch.cuda.stream(stream):
            big.set_surrogate(mlp, info["f_scale"], info["threshold"], mlp.bounds)
            nb = 4
            ms, got, fall = _time_modes(big, modes, nb, 2, mlp.bounds)
        torch.cuda.synchronize(dev)
        out["large_tank"] = {"workload": f"{nb * big.n_boid:,} queries: {nb} states x {big.n_boid:,} boids of the "
                                         "settled 2,097,152-particle tank (trained on the column: a shift)",
                             "queries": nb * big.n_boid}
        out["large_tank"].update(_mode_report(surrogate, ms, got, fall, nb * big.n_boid, nb))
    return out


def run_mlp_throughput(a):
    """Forward passes of the surrogate network on 65,536 feature rows (the
    1,024 boid rows of a column state, tiled 64 times): queries per second
    and the tensor rate of the four layers, per CUDA events."""
    import torch

    from paper_2311_15088_gb300 import surrogate
    from paper_2311_15088_gb300.sph import Mlp, Scene

    sc = scenes.dam_break_column(seed_offset=140)
    p = _params(sc)
    s = Scene(p, len(sc["fluid_pos"]), len(sc["boid_pos"]))
    s.set_state(sc["fluid_pos"], sc["fluid_vel"], sc["boid_pos"], sc["boid_vel"])
    s.step(3)
    X = s.features().repeat(64, 1).contiguous()
    m = Mlp(X.shape[0])
    m.set_params(torch.from_numpy(surrogate.init_params(0)))
    for _ in range(max(a.warmup, 3)):
        m.forward(X)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(a.steps):
        m.forward(X)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / a.steps
    flops = 2.0 * X.shape[0] * (272 * 256 + 256 * 256 * 2 + 256 * 16)
    print(json.dumps({"metric": "surrogate MLP forward, queries/s", "value": X.shape[0] / (ms * 1e-3),
                      "unit": "queries/s", "ms_per_batch": ms, "batch": int(X.shape[0]), "steps": a.steps,
                      "tflops": flops / (ms * 1e-3) / 1e12, "status": m.status()}), flush=True)
    return 0


# ---------------------------------------------------------------- arms

def run_reference(a):
    world, rank, _ = _dist()
    if rank != 0:
        return 0
    sc, desc, _settle = _workload(a.workload)
    p = dict(sc["params"])
    if p.get("mass") is None:
        import oracle

        p["mass"] = float(np.float32(oracle.lattice_mass(p, sc["lattice_spacing"])))
    fp, fv, bp, bv = sc["fluid_pos"], sc["fluid_vel"], sc["boid_pos"], sc["boid_vel"]
    per_step = a.reference_budget / max(a.steps + a.warmup, 1)
    # warm-up sample steps are part of the budget but not of the figure
    if a.warmup:
        _oracle_rate(p, fp, fv, bp, bv, per_step, steps=a.warmup)
    rate, cores, sdesc, steps, npart, el = _oracle_rate(p, fp, fv, bp, bv, per_step, steps=a.steps)
    line = {
        "impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": a.gpus,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * el / max(steps, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": desc + " (initial state: the oracle does not settle it)"},
        "cpu_baseline": {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sdesc,
                         "cpu": _cpu_model(), "host_cpus": os.cpu_count()},
        "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(a):
    import torch

    from paper_2311_15088_gb300 import sph
    from paper_2311_15088_gb300.sph import Scene

    world, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    _set_fp32_peak(dev)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    sc, desc, settle = _workload(a.workload)
    if a.settle is not None and settle:
        settle = a.settle
        desc = desc.replace(f"settled {SETTLE} steps", f"settled {settle} steps")
    p = _params(sc)
    if a.cell_x is not None:
        p["cell_size_x"] = float(np.float32(np.float32(p["h"]) * np.float32(a.cell_x)))
    nf, nb = len(sc["fluid_pos"]), len(sc["boid_pos"])
    z = np.zeros((0, 4), np.float32)

    # settle the fluid alone, then release the boids
    if settle:
        s0 = Scene(p, nf, 0, device=dev)
        s0.set_state(sc["fluid_pos"], sc["fluid_vel"], z, z)
        s0.step(settle)
        fp, fv, _, _ = s0.get_state()
        del s0
    else:
        fp, fv = sc["fluid_pos"], sc["fluid_vel"]
    s = Scene(p, nf, nb, device=dev)
    s.set_state(fp, fv, sc["boid_pos"], sc["boid_vel"])
    for _ in range(a.warmup):
        s.step(1)
    torch.cuda.synchronize(dev)
    work0 = _work_snapshot(s)
    if a.neighbor_lists:
        s.set_neighbor_lists(3 * work0["pairs"])
    start_state = [t.clone() for t in s.get_state()]  # the e2e leg restarts from here

    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(a.steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(a.steps)]
    sph.sph_profile_enable(s.handle, a.steps * len(sph.KINDS) + 16)
    clocks = ClockSampler(local)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    launches0 = s.launches
    # the work of a step grows as the fluid compresses: sample the candidate
    # and neighbour counts between timed steps (outside the step events)
    every = max(1, a.steps // 20)
    works = []
    for k in range(a.steps):
        flush.zero_()
        ev0[k].record()
        s.step(1)
        ev1[k].record()
        if k % every == every - 1:
            works.append(_work_snapshot(s))
    torch.cuda.synchronize(dev)
    if world > 1:
        torch.distributed.barrier()
    launches = s.launches - launches0
    clk = clocks.stop()
    prof = sph.sph_profile_read(s.handle)
    sph.sph_profile_enable(s.handle, 0)
    step_ms = [e0.elapsed_time(e1) for e0, e1 in zip(ev0, ev1)]
    t = _max_over_ranks(sum(step_ms) / 1e3, world, dev)
    value = _job_value(nf, a.steps, world, t)
    work1 = _work_snapshot(s)
    status = s.status()

    # ---- roofline of the dominant pass and the HBM view of the step
    works = works or [work0, work1]
    cand = statistics.mean(w["candidates"] for w in works)
    pairs = statistics.mean(w["pairs"] for w in works)
    over = statistics.mean(w["overflow_candidates"] for w in works)
    n_all = nf + nb
    passes = {k: {"ms_per_step": ms / max(cnt, 1), "launch_groups": cnt} for k, (ms, cnt) in prof.items() if cnt}
    if nb:
        passes["note"] = ("boid_bin and boid_rules (F_b + rules) run on the step's side stream alongside the "
                          "fluid passes: their times are spans that overlap density and forces")
    f_ms = passes["forces"]["ms_per_step"]
    d_ms = passes["density"]["ms_per_step"]
    stencil = STENCIL_CAND_PER_NBR * pairs
    force_flops = FLOP_CAND * stencil + FLOP_FORCE_PAIR * pairs
    dens_flops = FLOP_CAND * stencil + FLOP_DENS_PAIR * (pairs + n_all)
    segs = statistics.mean(w["segments"] for w in works)
    if s.tuning[1]:  # segments: stored pairs (self included) + overflow tests
        force_exec = FLOP_FORCE_PAIR * (pairs + nf) + FLOP_CAND * over
    else:
        force_exec = FLOP_CAND * cand + FLOP_FORCE_PAIR * pairs
    dens_exec = FLOP_CAND * cand + FLOP_DENS_PAIR * (pairs + n_all)
    achieved = force_flops / (f_ms * 1e-3) / 1e12
    src_sha = _source_sha(*(os.path.join(ROOT, "paper_2311_15088_gb300", "csrc", f)
                            for f in ("sph_physics.cu", "sph_internal.cuh")))
    traffic = {k: v["bytes"] for k, v in KERNEL_TRAFFIC.items() if v.get("source_sha256") == src_sha}
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    hbm_src = "measured" if "hbm_gbs" in peaks else "fallback"
    ncells = s.dims[0] * s.dims[1] * s.dims[2]
    step_bytes = n_all * sum(BYTES.values()) + ncells * BYTES_PER_CELL_SCAN
    ms_per_step = 1e3 * t / a.steps
    hbm_pass = {}
    for k in ("scatter", "sort", "density", "forces"):
        if k in passes:
            gbs = n_all * BYTES[k] / (passes[k]["ms_per_step"] * 1e-3) / 1e9
            hbm_pass[k] = {"GB/s": gbs, "frac": gbs / hbm_peak}
    both = (force_flops + dens_flops) / ((f_ms + d_ms) * 1e-3) / 1e12
    roofline = {
        "bound": "alu", "kernel": "k_forces (pair forces + integration)", "achieved": achieved,
        "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP32_PEAK_TFLOPS,
        "traffic": traffic.get("k_forces"),
        "peak_source": FP32_PEAK_SOURCE,
        "flops_per_launch": force_flops,
        "flops_definition": "27-cell stencil at cell size h: 9 flops x 27/(4pi/3) x neighbours + 35 x neighbours",
        "executed": {"flops_per_launch": force_exec, "achieved": force_exec / (f_ms * 1e-3) / 1e12,
                     "frac": force_exec / (f_ms * 1e-3) / 1e12 / FP32_PEAK_TFLOPS,
                     "definition": "35 x stored pairs (self included) + 9 x candidates of overflowing particles"
                                   if s.tuning[1] else "9 x candidates + 35 x pairs",
                     "candidates_per_particle": cand / n_all,
                     "segments_per_particle": segs / n_all,
                     "overflow_particles": statistics.mean(w["overflow_particles"] for w in works)},
        "density_pass": {"achieved": dens_flops / (d_ms * 1e-3) / 1e12,
                         "frac": dens_flops / (d_ms * 1e-3) / 1e12 / FP32_PEAK_TFLOPS,
                         "executed_frac": dens_exec / (d_ms * 1e-3) / 1e12 / FP32_PEAK_TFLOPS,
                         "traffic": traffic.get("k_density")},
        "neighbour_passes": {"achieved": both, "frac": both / FP32_PEAK_TFLOPS,
                             "definition": "both passes' algorithmic flops over their summed time (the density "
                                           "pass tests the candidates once for both)"},
    }
    hbm = {"algorithmic_bytes_per_step": step_bytes, "achieved_GBps": step_bytes / (ms_per_step * 1e-3) / 1e9,
           "peak_GBps": hbm_peak, "frac": step_bytes / (ms_per_step * 1e-3) / 1e9 / hbm_peak,
           "peak_source": hbm_src, "per_pass": hbm_pass}

    # ---- end to end through host buffers, from the state the timed steps
    # started at: each step uploads the state from pinned host memory, steps
    # and downloads the new state
    host = [t.cpu().pin_memory() for t in start_state]
    torch.cuda.synchronize(dev)
    n_e2e = a.steps if a.e2e_steps is None else min(a.e2e_steps, a.steps)
    t0 = time.perf_counter()
    for _ in range(n_e2e):
        s.set_state_host(*host)
        s.step(1)
        s.get_state_host(host)
    e2e_t = time.perf_counter() - t0
    e2e = {"value": nf * n_e2e * world / e2e_t, "unit": UNIT,
           "h2d_bytes_per_step": int(sum(h.numel() * 4 for h in host)),
           "d2h_bytes_per_step": int(sum(h.numel() * 4 for h in host)), "steps": n_e2e,
           "device_ms_same_steps": sum(step_ms[:n_e2e]), "wall_ms": 1e3 * e2e_t}

    # ---- CPU oracle on a bounded sample of the same (settled) workload
    cpu = None
    if world == 1 and rank == 0 and not a.no_cpu_baseline:
        st = [x.cpu().numpy() if hasattr(x, "cpu") else x for x in s.get_state()]
        rate, cores, sdesc, _steps, _np, _el = _oracle_rate(p, *st, step_seconds=a.cpu_seconds / 3,
                                                            min_seconds=a.cpu_seconds)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sdesc,
               "cpu": _cpu_model(), "host_cpus": os.cpu_count()}

    nsearch = _neighbor_search(s, dev)
    surface = None if a.no_surface else _surface(s, dev, p, a.warmup)
    batched = None if a.no_batch else run_batched(a, dev, flush)
    sur = None if a.no_surrogate else run_surrogate(a, dev, big=s)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": desc, "fluid_particles": nf, "boids": nb, "settle_steps": settle,
                       "l2": "flushed between timed steps (256 MiB write outside the step events)",
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "cell_size_over_h": float(np.float32(p["cell_size"]) / np.float32(p["h"])),
                       "cell_size_x_over_h": float(np.float32(p.get("cell_size_x") or p["cell_size"])
                                                   / np.float32(p["h"])),
                       "tuning": {"block": s.tuning[0], "use_segments": s.tuning[1], "ppt": s.ppt},
                       "force_pass_neighbours": "pair lists" if a.neighbor_lists else "walk",
                       "neighbours_mean": statistics.mean(w["nbr_mean"] for w in works),
                       "neighbours_max": max(w["nbr_max"] for w in works),
                       "candidates_per_particle": cand / n_all},
            "diagnostics": {"source": "sph_stats (fluid particles) after the first and the last sampled timed step",
                            "first": works[0]["stats"], "last": works[-1]["stats"]},
            "roofline": roofline, "hbm": hbm, "passes": passes, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": launches, "clocks": clk, "device_status": status, "neighbor_search": nsearch,
            "batched": batched,
            "surrogate": sur,
            "surface": surface,
            "step_ms": {"min": min(step_ms), "median": statistics.median(step_ms), "max": max(step_ms)},
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    a = _args()
    if a.impl == "reference":
        return run_reference(a)
    if a.mlp_throughput:
        return run_mlp_throughput(a)
    return run_ours(a)


if __name__ == "__main__":
    sys.exit(main())
