#!/usr/bin/env python
"""Benchmark of the GB300 GRMHD RK stage: FP64 zone-updates per second per RK stage.

Workload: the 256^3 block of the rotating magnetised torus with an axial jet (Lorentz factor up to 7) in the
frozen isotropic Schwarzschild slice (M = 0.1, centre at (-1, 0, 0)), WENO-Z + HLLE + UCT, ideal gas Gamma = 4/3,
copy BCs, atmosphere floor 1e-10; one step = one classical RK4 step (4 stages: ghost fill, recovery,
reconstruction, face solve, UCT, potentials, sources, combine).  Inputs are seeded and synthetic; the
frozen-metric geometry is derived once before timing (asterx_prepare).  The state lives in HBM (about 1.3 GB per
state copy and 32 GB of workspace, far above the 129 MB L2), so no L2 flush is needed.  The 128^3 block of
Balsara test-1 states in the same slice (WENO-Z, Gamma = 5/3) is timed beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 it is launched by torch.distributed.run; every rank runs an independent replica of the block
(no data exchange: the path has none) and rank 0 prints one JSON line.  --impl reference times the CPU oracle
(the reference implementation of this tier) on all host cores on a bounded slab of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import platform
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "FP64 GRMHD zone-updates/s per RK stage; batched-vs-single and adjoint/forward time"
UNIT = "zone-updates/s"
WORKLOAD = ("256^3 block + 3 ghosts, FP64, ideal gas Gamma=4/3, WENO-Z + HLLE + UCT, Noble2D/Palenzuela c2p, "
            "rotating magnetised torus rho=max(1e-2 exp(-(R-0.3)^2/0.01-z^2/0.01),1e-10), p=0.1 rho^(4/3), "
            "Omega=0.5, axial jet W<=7 (seed 105), frozen isotropic Schwarzschild M=0.1 centred 0.5 outside the "
            "box, copy BCs, one RK4 step = 4 stages")
WORKLOAD_128 = ("128^3 block + 3 ghosts, FP64, Gamma=5/3, WENO-Z + HLLE + UCT, Balsara-1 Riemann data split at x=0 "
                "(Bx=0.5, By=+-1), frozen isotropic Schwarzschild M=0.1 (seed 102)")
# kernels the library launches per RK stage: 3 + 3 ghost sweeps, 2 field kernels, recovery, velocity, 3 x
# (reconstruction + face solve), vertex potentials, 3 edge kernels, scalar potential, cells
LAUNCHES_PER_STAGE = 28
# FP64 units: 2 DFMA per clock per SM (GB300), 2 flops each
DFMA_PER_CLOCK_PER_SM = 2


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--n", type=int, default=256, help="cells per axis of the torus block (default: the 256^3 workload)")
    ap.add_argument("--balsara-n", type=int, default=128,
                    help="cells per axis of the Balsara block (timed beside the torus; also the tiled and "
                         "two-level measurements)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the uneven-batch measurement")
    ap.add_argument("--batch-blocks", type=int, default=512)
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint-vs-forward measurement")
    ap.add_argument("--no-balsara", action="store_true",
                    help="skip the 128^3 Balsara block (and the tiled and two-level runs measured against it)")
    ap.add_argument("--adjoint-n", type=int, default=64, help="cells per axis of the adjoint workload")
    ap.add_argument("--no-refined", action="store_true",
                    help="skip the two-level (refined box) measurement")
    ap.add_argument("--no-tiled", action="store_true",
                    help="skip the tiled-domain (ghost exchange between blocks) measurement")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the Lax-Friedrichs / flux-CT / RK2 step measurements")
    ap.add_argument("--no-coupling", action="store_true",
                    help="skip the stress-energy tensor and time-dependent-metric step measurements")
    ap.add_argument("--profile-region", choices=("none", "forward", "adjoint", "batched", "coupling", "tiled", "refined",
                                                  "subcycled"), default="none",
                    help="bracket one extra forward RK4 step (main workload), one adjoint step, one batched "
                         "step and one step of the equal-volume block, one geometry derivation and one "
                         "stress-energy tensor call, one step of the 4x4x4-tiled domain, one two-level step or "
                         "one subcycled two-level step with cudaProfilerStart/Stop, for a profiler run with "
                         "--profile-from-start off")
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_rate(world, cells, steps, ms_max):
    """Whole-job zone-updates/s per RK stage: every rank advances its own replica of `cells` interior cells by
    `steps` RK4 steps (4 stages each); the slowest rank's time (ms, max over ranks) is the job's."""
    return world * cells * 4 * steps / (ms_max / 1e3)


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


class ClockSampler:
    """nvidia-smi sampled every 200 ms during the timed region (SM clock, max clock, power, throttle reasons)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = sorted(float(r[1]) for r in rows if r[1].replace(".", "").isdigit())
        smax = max((float(r[2]) for r in rows if r[2].replace(".", "").isdigit()), default=None)
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        power = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": smax, "reasons": reasons,
                "samples": len(rows), "power_w_max": max(power) if power else None}


def read_kv(name):
    """key = value lines of a committed profile summary (None if the file is absent)."""
    path = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(path):
        return None
    vals = {}
    with open(path) as f:
        for line in f:
            if "=" in line and not line.startswith("#"):
                k, v = line.split("=", 1)
                vals[k.strip()] = float(v.split()[0])
    return vals


def read_stage_flops(n):
    """Algorithmic FP64 flops per zone-stage and per kernel unit on the n^3 torus-and-jet workload, counted by the
    oracle's flop-counting scalar (written by oracle/count_stage_flops.py)."""
    return read_kv(f"stage_flops_torus_jet_{n}.txt")


def read_traffic(n):
    """DRAM bytes of one face-solve launch on the n^3 torus workload (from an ncu capture, scaled by faces)."""
    v = read_kv(f"faces_torus_jet_{n}_traffic.txt")
    return v.get("dram_bytes_per_launch") if v else None


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                name = line.split(":", 1)[1].strip()
                if name and name != "-":
                    return name
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                low = line.lower()
                if low.startswith("model name") or low.startswith("cpu part") or low.startswith("hardware"):
                    name = line.split(":", 1)[1].strip()
                    if name:
                        return name
    except OSError:
        pass
    return platform.processor() or platform.machine()


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def slab_workload(w_full, ny, nz):
    from paper_2406_11669_gb300 import workloads as W
    n = w_full.n
    lo = (0, (n[1] - ny) // 2, (n[2] - nz) // 2)
    return W.sub_block(w_full, lo, (n[0], ny, nz), name="slab")


def cpu_oracle_steps(w, steps, threads):
    """Times `steps` oracle RK4 steps on workload w with `threads` OpenMP threads; returns (seconds per step,
    threads in effect)."""
    import oracle as O
    used = O.set_threads(threads)
    U, P = O.initial_state(w)
    M = O.metric_array(w)
    O.ghost_fill_state(w, U)
    t0 = time.perf_counter()
    for _ in range(steps):
        U, _ = O.rk4_step(w, M, U, P)
        O.ghost_fill_state(w, U)
    return (time.perf_counter() - t0) / steps, used


def cpu_baseline(w_full):
    """The oracle as it stands on the host: one RK4 step of a central x-slab of the workload on one core, and of a
    wider slab on every core (OpenMP over (k, j) pencils)."""
    model, cores = cpu_model(), host_cores()
    out = {"kind": "oracle", "unit": UNIT, "cpu_model": model, "nproc": cores}
    runs = []
    for threads, ny in ((1, 8), (cores, 24)):
        w = slab_workload(w_full, ny, ny)
        sec, used = cpu_oracle_steps(w, 1, threads)
        cells = w.interior_cells
        runs.append({"cores": used, "value": cells * 4 / sec, "seconds": sec,
                     "sample": f"one RK4 step of the central {w.n[0]}x{ny}x{ny} x-slab of the workload ({cells} "
                               f"cells) on {used} thread(s), g++ -O2 -fopenmp"})
    out["one_core"], out["all_cores"] = runs
    out["value"] = runs[1]["value"]
    out["cores"] = runs[1]["cores"]
    out["sample"] = runs[1]["sample"] + f"; one core: {runs[0]['value']:.4g} {UNIT}"
    return out


def _upload_block(w, dev):
    import numpy as np
    import torch

    from paper_2406_11669_gb300 import workloads as W
    M = torch.from_numpy(np.ascontiguousarray(np.stack([w.metric[k] for k in W.METRIC_NAMES]))).to(dev)
    P = torch.from_numpy(np.ascontiguousarray(np.stack([w.prims[k] for k in W.PRIM_NAMES]))).to(dev)
    U = torch.zeros((9,) + w.shape, dtype=torch.float64, device=dev)
    U[5] = torch.from_numpy(w.A["Ax"]).to(dev)
    U[6] = torch.from_numpy(w.A["Ay"]).to(dev)
    U[7] = torch.from_numpy(w.A["Az"]).to(dev)
    U[8] = torch.from_numpy(w.Psi).to(dev)
    return M, U, P


def counters(t):
    c = t.cpu().tolist()
    return {"n_noble": c[0], "n_fallback": c[1], "n_atm": c[2], "n_failed": c[3], "noble_iters": c[4]}


def run_batched(args, dev, stream):
    """Uneven batch of the magnetised-star workload (512 blocks, n per axis in {16,24,32,48,64}, dx = 1/256,
    PPM, Schwarzschild M = 0.2) in one batched step, against one block of equal total interior volume with the
    same physics and generator.  Returns the rates (zone-updates/s per RK stage) and their ratio."""
    import torch

    from paper_2406_11669_gb300 import asterx as A
    from paper_2406_11669_gb300 import workloads as W

    lay = W.star_layout(nblocks=args.batch_blocks)
    entries = []
    cells = 0
    for n, o in lay:
        w = W.star_block(n, o)
        M, U, P = _upload_block(w, dev)
        entries.append((w.n, w.g, w.x0, w.dx, w.bc, M, U, P))
        cells += w.interior_cells
        params, dt = w.params, w.dt
    batch = A.Batch(params, entries, device=dev)
    batch.prepare()
    batch.prim2con()
    steps = max(1, min(args.steps, 3))
    batch.step(dt, nsteps=1)
    torch.cuda.synchronize(dev)
    stats_b = torch.zeros(5, dtype=torch.int64, device=dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    batch.step(dt, nsteps=steps, stats=stats_b)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms_b = e0.elapsed_time(e1) / steps
    if args.profile_region == "batched":
        torch.cuda.profiler.start()
        batch.step(dt, nsteps=1)
        torch.cuda.synchronize(dev)
        torch.cuda.profiler.stop()
    pool_bytes = batch.ws_bytes
    del batch
    torch.cuda.empty_cache()
    # the same blocks stepped one at a time through the single-block path (one launch sequence per block, as a
    # code that loops over its blocks does): the sum of the blocks' step times
    loop_ms = 0.0
    for (n, g, x0, dx_, bc, M, U, P) in entries:
        sb = A.Solver(params, n, g, x0, dx_, bc, device=dev)
        sb.prepare(M)
        sb.rk4_step(U, P, dt)  # warm-up (and the autotuner's first launch at this size)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        sb.rk4_step(U, P, dt)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        loop_ms += e0.elapsed_time(e1)
        del sb
    del entries
    torch.cuda.empty_cache()
    # one block of the same total interior volume, centred on the star
    side = int(round(cells ** (1.0 / 3.0)))
    h = 1.0 / 256.0
    w = W.star_block((side, side, side), (-0.5 * side * h,) * 3)
    M, U, P = _upload_block(w, dev)
    s = A.Solver.for_workload(w, device=dev)
    s.prepare(M)
    s.fill_ghosts(U)
    s.prim2con(U, P)
    s.rk4_step(U, P, w.dt)
    torch.cuda.synchronize(dev)
    stats_s = torch.zeros(5, dtype=torch.int64, device=dev)
    e0.record(stream)
    for _ in range(steps):
        s.rk4_step(U, P, w.dt, stats=stats_s)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms_s = e0.elapsed_time(e1) / steps
    if args.profile_region == "batched":
        torch.cuda.profiler.start()
        s.rk4_step(U, P, w.dt)
        torch.cuda.synchronize(dev)
        torch.cuda.profiler.stop()
    single_cells = w.interior_cells
    del s, M, U, P
    torch.cuda.empty_cache()
    rate_b = cells * 4 / (ms_b / 1e3)
    rate_s = single_cells * 4 / (ms_s / 1e3)
    return {"workload": f"{len(lay)} uneven blocks (n per axis in 16..64, seed 103), magnetised star, PPM, "
                        f"Schwarzschild M=0.2, one batched launch per kernel",
            "blocks": len(lay), "interior_cells": cells, "value": rate_b, "unit": UNIT, "ms_per_step": ms_b,
            "steps": steps, "pool_bytes": int(pool_bytes),
            "c2p_counters": counters(stats_b),
            "per_block_loop": {"ms_per_step": loop_ms, "value": cells * 4 / (loop_ms / 1e3),
                               "batched_vs_loop": loop_ms / ms_b},
            "single_equal_volume": {"n": side, "interior_cells": single_cells, "value": rate_s, "ms_per_step": ms_s,
                                    "c2p_counters": counters(stats_s)},
            "batched_vs_single": rate_b / rate_s}


def run_tiled(args, dev, stream, single_ms):
    """The 128^3 Balsara domain cut into 2x2x2 blocks of 64^3 and 4x4x4 blocks of 32^3, advanced by the batched
    launch with same-level ghost exchange between the blocks, against the single 128^3 block (single_ms)."""
    import numpy as np
    import torch

    from paper_2406_11669_gb300 import asterx as A
    from paper_2406_11669_gb300 import workloads as W

    w = W.balsara_schwarzschild(n=(args.balsara_n,) * 3)
    M, U, P = _upload_block(w, dev)
    out = {}
    for k in (2, 4):
        m = args.balsara_n // k
        cuts = [list(range(0, args.balsara_n + 1, m))] * 3
        entries = []
        for bz in range(k):
            for by in range(k):
                for bx in range(k):
                    lo = (bx * m, by * m, bz * m)
                    sl = (slice(None),) + tuple(slice(lo[d], lo[d] + m + 2 * w.g + 1) for d in (2, 1, 0))
                    x0 = tuple(w.x0[d] + lo[d] * w.dx[d] for d in range(3))
                    entries.append(((m, m, m), w.g, x0, w.dx, w.bc, M[sl].contiguous(), U[sl].contiguous(),
                                    P[sl].contiguous()))
        batch = A.Batch(w.params, entries, device=dev, tiling=((k, k, k), cuts))
        batch.prepare()
        batch.prim2con()
        steps = max(1, min(args.steps, 3))
        batch.step(w.dt, nsteps=1)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        batch.step(w.dt, nsteps=steps)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / steps
        if args.profile_region == "tiled" and k == 4:
            torch.cuda.profiler.start()
            batch.step(w.dt, nsteps=1)
            torch.cuda.synchronize(dev)
            torch.cuda.profiler.stop()
        finite = all(bool(torch.isfinite(e[6]).all()) for e in entries)
        batch.release()
        del batch, entries
        torch.cuda.empty_cache()
        out[f"{k}x{k}x{k}"] = {"block_n": m, "ms_per_step": ms, "value": w.interior_cells * 4 / (ms / 1e3),
                               "unit": UNIT, "tiled_vs_single": single_ms / ms, "finite": finite}
    del M, U, P
    torch.cuda.empty_cache()
    return out


def run_refined(args, dev, stream, single_ms):
    """Two refinement levels on the 128^3 Balsara workload: the 128^3 block plus a fine block of half the spacing over
    its central 64^3 coarse cells (128^3 fine cells; fine data prolonged from the coarse level, the Schwarzschild
    metric evaluated at the fine vertices), stepped together with the fine time step (prolongation of each coarse
    stage state to the fine ghosts, restriction after the step).  Compared with two plain steps of 128^3 blocks.
    Then the same levels subcycled: one coarse step of twice the size, two fine steps, against two of the steps
    with the fine step on both levels (the same time covered)."""
    import numpy as np
    import torch

    from paper_2406_11669_gb300 import asterx as A
    from paper_2406_11669_gb300 import workloads as W

    w = W.balsara_schwarzschild(n=(args.balsara_n,) * 3)
    M, U, P = _upload_block(w, dev)
    sc = A.Solver.for_workload(w, device=dev)
    sc.prepare(M)
    sc.fill_ghosts(U)
    sc.prim2con(U, P)
    Lc, m = args.balsara_n // 4, args.balsara_n // 2
    nf = (2 * m,) * 3
    x0f = tuple(w.x0[d] + Lc * w.dx[d] for d in range(3))
    dxf = tuple(h / 2 for h in w.dx)
    Nf = [v + 2 * w.g for v in nf]
    shape_f = (Nf[2] + 1, Nf[1] + 1, Nf[0] + 1)
    Xv, Yv, Zv = W.positions(nf, w.g, x0f, dxf, W.VERTEX)
    metf = W.schwarzschild_isotropic(Xv, Yv, Zv, 0.1, (-1.0, 0.0, 0.0), shape_f)
    Mf = torch.from_numpy(np.ascontiguousarray(np.stack([metf[k] for k in W.METRIC_NAMES]))).to(dev)
    sf = A.Solver(w.params, nf, w.g, x0f, dxf, w.bc, device=dev)
    sf.prepare(Mf)
    Uf, Pf = sf.zeros_state(), sf.zeros_prims()
    A.prolong(sc, sf, U, P, Uf, Pf, all_points=True)
    dt = 0.5 * w.dt
    A.rk4_step_refined(sc, sf, U, P, Uf, Pf, dt)
    torch.cuda.synchronize(dev)
    steps = max(1, min(args.steps, 3))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        A.rk4_step_refined(sc, sf, U, P, Uf, Pf, dt)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / steps
    if args.profile_region == "refined":
        torch.cuda.profiler.start()
        A.rk4_step_refined(sc, sf, U, P, Uf, Pf, dt)
        torch.cuda.synchronize(dev)
        torch.cuda.profiler.stop()
    # subcycled: one coarse step of twice the fine step, two fine steps (the same time covered as two of the
    # steps above)
    A.rk4_step_subcycled(sc, sf, U, P, Uf, Pf, 2.0 * dt)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    for _ in range(steps):
        A.rk4_step_subcycled(sc, sf, U, P, Uf, Pf, 2.0 * dt)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms_sub = e0.elapsed_time(e1) / steps
    if args.profile_region == "subcycled":
        torch.cuda.profiler.start()
        A.rk4_step_subcycled(sc, sf, U, P, Uf, Pf, 2.0 * dt)
        torch.cuda.synchronize(dev)
        torch.cuda.profiler.stop()
    finite = bool(torch.isfinite(U).all()) and bool(torch.isfinite(Uf).all())
    cells = w.interior_cells + int(np.prod(nf))
    updates_sub = 4 * w.interior_cells + 8 * int(np.prod(nf))  # zone-stage updates per coarse step
    del sc, sf, M, U, P, Mf, Uf, Pf
    torch.cuda.empty_cache()
    return {"coarse_n": args.balsara_n, "fine_box_coarse_cells": m, "fine_n": nf[0], "ms_per_step": ms,
            "value": cells * 4 / (ms / 1e3), "unit": UNIT, "vs_two_single_steps": 2.0 * single_ms / ms,
            "finite": finite,
            "subcycled": {"ms_per_coarse_step": ms_sub, "value": updates_sub / (ms_sub / 1e3), "unit": UNIT,
                          "speedup_vs_same_step": 2.0 * ms / ms_sub}}


def run_adjoint(args, dev, stream):
    """The adjoint workload (64^3 periodic, weak-field lapse, PPM): time of one RK4 step forward against one
    adjoint RK4 step (forward recompute of the four stage states from the checkpoint, then the four reversed
    stages); then the whole gradient of J = 1/2 sum (D~_10 - T)^2 with respect to the initial primitives and
    potentials (10 checkpointed steps forward, 10 adjoint steps, adjoint of the initial data; one untimed
    evaluation first)."""
    import numpy as np
    import torch

    from paper_2406_11669_gb300 import asterx as A
    from paper_2406_11669_gb300 import workloads as W

    w = W.weak_field_modes(n=(args.adjoint_n,) * 3)
    M, U, P = _upload_block(w, dev)
    s = A.Solver.for_workload(w, device=dev)
    s.prepare(M)
    s.fill_ghosts(U)
    s.prim2con(U, P)
    U0, P0 = U.clone(), P.clone()
    lam = torch.zeros_like(U)
    g = w.g
    inter = (slice(g, g + w.n[2]), slice(g, g + w.n[1]), slice(g, g + w.n[0]))
    lam[(0,) + inter] = 1e-3
    reps = max(1, min(args.steps, 5))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    # warm-up both directions (allocates the adjoint workspace)
    s.rk4_step(U, P, w.dt)
    s.rk4_step_adjoint(U0, P, lam, w.dt)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    for _ in range(reps):
        s.rk4_step(U, P, w.dt)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms_f = e0.elapsed_time(e1) / reps
    e0.record(stream)
    for _ in range(reps):
        s.rk4_step_adjoint(U0, P, lam, w.dt)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms_a = e0.elapsed_time(e1) / reps
    if args.profile_region == "adjoint":
        torch.cuda.profiler.start()
        s.rk4_step_adjoint(U0, P, lam, w.dt)
        torch.cuda.synchronize(dev)
        torch.cuda.profiler.stop()
    # whole 10-step gradient
    nsteps = 10
    T = torch.from_numpy(W.weak_field_target(w)).to(dev)
    ckpt = [torch.empty_like(U) for _ in range(nsteps)]
    lamP = torch.zeros_like(P)

    def gradient():
        U.copy_(U0)
        P.copy_(P0)
        s.rk4_steps_checkpointed(U, P, w.dt, ckpt)
        lam.zero_()
        lam[(0,) + inter] = U[(0,) + inter] - T[inter]
        s.rk4_adjoint_steps(ckpt, P, lam, w.dt)
        s.prim2con_adjoint(U0, P0, lam, lamP)

    gradient()  # warm-up: the first use of torch's own kernels for the loss seed loads them
    torch.cuda.synchronize(dev)
    e0.record(stream)
    gradient()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms_grad = e0.elapsed_time(e1)
    grad_finite = bool(torch.isfinite(lamP).all()) and bool(torch.isfinite(lam).all())
    grad_norm = float(lamP[0][inter].abs().max())
    ckpt_bytes = nsteps * U.numel() * 8
    del ckpt, s, U, P, U0, P0, lam, lamP, M
    torch.cuda.empty_cache()
    return {"workload": f"{w.n[0]}^3 periodic, lapse 1 - 0.01 sin 2 pi x, PPM (seed 104)",
            "forward_ms_per_step": ms_f, "adjoint_ms_per_step": ms_a, "adjoint_vs_forward": ms_a / ms_f,
            "steps_timed": reps,
            "gradient_10_steps": {"ms": ms_grad, "checkpoint_bytes": ckpt_bytes, "finite": grad_finite,
                                  "max_abs_dJ_drho": grad_norm}}


def run_coupling(args, s, U, P, M, w, dev, stream):
    """Coupling to a spacetime solver on the benchmark block: T_{mu nu} at the (n+1)^3 owned vertices (asterx_tmunu:
    face and centre field, u = W v, then the vertex kernel), and one RK4 step whose four stages each re-derive the
    geometry from a stage metric (asterx_rk4_step_metrics) against the frozen-metric step."""
    import torch

    T = torch.zeros((10,) + tuple(U.shape[1:]), dtype=torch.float64, device=dev)
    reps = max(3, min(args.steps * 4, 20))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.tmunu(U, P, T)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    for _ in range(reps):
        s.tmunu(U, P, T)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms_t = e0.elapsed_time(e1) / reps
    if args.profile_region == "coupling":
        torch.cuda.profiler.start()
        s.prepare(M)
        s.tmunu(U, P, T)
        torch.cuda.synchronize(dev)
        torch.cuda.profiler.stop()
    finite = bool(torch.isfinite(T).all())
    del T
    s.prepare(M)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    for _ in range(reps):
        s.prepare(M)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms_prep = e0.elapsed_time(e1) / reps
    metrics = [M, M, M, M]
    s.rk4_step_metrics(U, P, w.dt, metrics)
    torch.cuda.synchronize(dev)
    steps = max(1, min(args.steps, 3))
    e0.record(stream)
    for _ in range(steps):
        s.rk4_step_metrics(U, P, w.dt, metrics)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms_dyn = e0.elapsed_time(e1) / steps
    e0.record(stream)
    for _ in range(steps):
        s.rk4_step(U, P, w.dt)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms_frozen = e0.elapsed_time(e1) / steps
    nv = 1
    for d in range(3):
        nv *= w.n[d] + 1
    return {"tmunu": {"vertices": nv, "ms": ms_t, "vertices_per_s": nv / (ms_t / 1e3), "finite": finite,
                      "launches": 4},
            "prepare_ms": ms_prep,
            "metric_step": {"ms_per_step": ms_dyn, "frozen_ms_per_step": ms_frozen,
                            "overhead": ms_dyn / ms_frozen - 1.0, "steps": steps}}


def run_variants(args, s, U, P, w, dev, stream, U0=None, P0=None):
    """The paper's alternative schemes on the benchmark block: one RK4 step with the Lax-Friedrichs flux, with flux
    constrained transport, with both, with the algebraic gauge, with MP5 and with PPM reconstruction, and one RK2
    step of the default scheme (rates per RK stage)."""
    import torch

    from paper_2406_11669_gb300 import asterx as A

    base = s.p
    out = {}
    steps = max(1, min(args.steps, 3))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    recon0 = s.params["recon"]
    for name, flux, efield, rk2, gauge, recon in (("lxf", 1, 0, False, 0, recon0), ("fct", 0, 1, False, 0, recon0),
                                                  ("lxf_fct", 1, 1, False, 0, recon0), ("rk2", 0, 0, True, 0, recon0),
                                                  ("algebraic_gauge", 0, 0, False, 1, recon0),
                                                  ("mp5", 0, 0, False, 0, 3), ("ppm", 0, 0, False, 0, 1)):
        s.p = A.params_struct(dict(s.params, flux=flux, efield=efield, gauge=gauge, recon=recon))
        step = s.rk2_step if rk2 else s.rk4_step
        if U0 is not None:  # every variant starts from the state the headline was timed on
            U.copy_(U0)
            P.copy_(P0)
        stats = torch.zeros(5, dtype=torch.int64, device=dev)
        step(U, P, w.dt)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        for _ in range(steps):
            step(U, P, w.dt, stats=stats)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / steps
        stages = 2 if rk2 else 4
        c = stats.cpu().tolist()
        out[name] = {"ms_per_step": ms, "value": w.interior_cells * stages / (ms / 1e3), "unit": UNIT,
                     "stages_per_step": stages, "steps": steps,
                     "c2p_counters": {"n_noble": c[0], "n_fallback": c[1], "n_atm": c[2], "n_failed": c[3]}}
    s.p = base
    return out


def run_reference(args):
    """The oracle as it stands, on every host core, each step one RK4 step of the central n x 16 x 16 x-slab of
    the workload (the slab crosses the jet and both sides of the torus)."""
    world, rank, _ = dist_env()
    if rank != 0:
        return
    from paper_2406_11669_gb300 import workloads as W
    w_full = W.torus_jet(n=(args.n,) * 3)
    w = slab_workload(w_full, 16, 16)
    del w_full
    cores = host_cores()
    if args.warmup > 0:
        cpu_oracle_steps(w, args.warmup, cores)
    sec, used = cpu_oracle_steps(w, args.steps, cores)
    cells = w.interior_cells
    value = cells * 4 / sec
    sample = (f"each step: one oracle RK4 step of the central {w.n[0]}x16x16 x-slab of the workload ({cells} "
              f"cells) on {used} host threads ({cpu_model()})")
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "sample_cells": cells},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": used, "kind": "oracle", "sample": sample,
                            "cpu_model": cpu_model(), "nproc": cores},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def time_steps(s, U, P, dt, steps, stream, dev, stats=None):
    """CUDA-event time (ms) of `steps` RK4 steps of solver s on the launching stream."""
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        s.rk4_step(U, P, dt, stats=stats)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    return e0.elapsed_time(e1)


def run_balsara(args, dev, stream):
    """The 128^3 Balsara block in the same slice (WENO-Z): rate per RK stage and its face-kernel launch time."""
    import torch

    from paper_2406_11669_gb300 import asterx as A
    from paper_2406_11669_gb300 import workloads as W

    w = W.balsara_schwarzschild(n=(args.balsara_n,) * 3)
    M, U, P = _upload_block(w, dev)
    s = A.Solver.for_workload(w, device=dev)
    s.prepare(M)
    s.fill_ghosts(U)
    s.prim2con(U, P)
    for _ in range(max(args.warmup, 1)):
        s.rk4_step(U, P, w.dt)
    torch.cuda.synchronize(dev)
    steps = max(3, args.steps)
    A.profile_enable(steps * 4 * 3)
    ms = time_steps(s, U, P, w.dt, steps, stream, dev)
    nface, face_ms = A.profile_read()
    A.profile_disable()
    del s, M, U, P
    torch.cuda.empty_cache()
    return {"workload": WORKLOAD_128, "ms_per_step": ms / steps, "steps": steps,
            "value": w.interior_cells * 4 * steps / (ms / 1e3), "unit": UNIT,
            "face_launch_ms": face_ms / max(nface, 1), "faces_per_launch": (w.n[0] + 1) * (w.n[0] ** 2 + 12 * w.n[0])}


def run_ours(args):
    import numpy as np
    import torch

    from paper_2406_11669_gb300 import asterx as A
    from paper_2406_11669_gb300 import workloads as W

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend="nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count

    w = W.torus_jet(n=(args.n,) * 3)
    s = A.Solver.for_workload(w, device=dev)
    M = torch.from_numpy(np.ascontiguousarray(np.stack([w.metric[k] for k in W.METRIC_NAMES]))).to(dev)
    P0 = np.ascontiguousarray(np.stack([w.prims[k] for k in W.PRIM_NAMES]))
    s.prepare(M)
    U = s.zeros_state()
    U[5] = torch.from_numpy(w.A["Ax"]).to(dev)
    U[6] = torch.from_numpy(w.A["Ay"]).to(dev)
    U[7] = torch.from_numpy(w.A["Az"]).to(dev)
    P = torch.from_numpy(P0).to(dev)
    del P0
    s.fill_ghosts(U)
    s.prim2con(U, P)
    stats = torch.zeros(5, dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream(dev)

    for _ in range(args.warmup):
        s.rk4_step(U, P, w.dt, stats=stats)
    torch.cuda.synchronize(dev)
    U_warm, P_warm = U.clone(), P.clone()  # the variants start from this state
    stats.zero_()
    A.profile_enable(args.steps * 4 * 3)
    barrier(world)
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    ms = time_steps(s, U, P, w.dt, args.steps, stream, dev, stats=stats)
    clk = clocks.stop()
    barrier(world)
    nface, face_ms = A.profile_read()
    A.profile_disable()
    ms_max = max_over_ranks(ms, world)
    cells = w.interior_cells
    value = replica_rate(world, cells, args.steps, ms_max)
    c2p = stats.cpu().tolist()
    if args.profile_region == "forward":
        torch.cuda.profiler.start()
        s.rk4_step(U, P, w.dt)
        torch.cuda.synchronize(dev)
        torch.cuda.profiler.stop()
    finite = bool(torch.isfinite(U[:, w.g:-w.g - 1, w.g:-w.g - 1, w.g:-w.g - 1]).all())

    # end to end through the host-buffer ABI call: H2D of U and P, the RK4 step, D2H of U and P, every step
    # (from the state the device-timed steps started from: the same K steps, since the cost of a step changes
    # as the torus evolves)
    hU = torch.empty(U.shape, dtype=torch.float64, pin_memory=True)
    hP = torch.empty(P.shape, dtype=torch.float64, pin_memory=True)
    dU2 = torch.empty_like(U)
    dP2 = torch.empty_like(P)
    hU.copy_(U_warm)
    hP.copy_(P_warm)
    s.rk4_step_host(hU, hP, dU2, dP2, w.dt)  # warm-up
    hU.copy_(U_warm)
    hP.copy_(P_warm)
    torch.cuda.synchronize(dev)
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        s.rk4_step_host(hU, hP, dU2, dP2, w.dt)
    e2e_s = max_over_ranks(time.perf_counter() - t0, world)
    e2e_value = world * cells * 4 * args.steps / e2e_s
    io_bytes = (9 + 5) * U[0].numel() * 8
    del hU, hP, dU2, dP2
    torch.cuda.empty_cache()

    # FP64 FMA throughput measured on this GPU: the peak of the roofline
    blocks, threads, iters = sms * 8, 256, 4096
    out = torch.empty(blocks * threads, dtype=torch.float64, device=dev)
    A.dfma_probe(out, blocks, threads, 64)
    torch.cuda.synchronize(dev)
    p0 = torch.cuda.Event(enable_timing=True)
    p1 = torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    A.dfma_probe(out, blocks, threads, iters)
    p1.record(stream)
    torch.cuda.synchronize(dev)
    dfma_tflops = blocks * threads * iters * 8 * 8 * 2 / (p0.elapsed_time(p1) / 1e3) / 1e12
    del out
    max_mhz = clk.get("sm_max_mhz") or 2070.0
    nominal_tflops = sms * DFMA_PER_CLOCK_PER_SM * 2 * max_mhz * 1e6 / 1e12

    if rank != 0:
        return
    faces_per_launch = (args.n + 1) * (args.n ** 2 + 12 * args.n)  # faces g..g+n, corner columns excluded
    sf = read_stage_flops(args.n) or {}
    flops_per_face = sf.get("face_solve_flops_per_face")
    face_avg_ms = face_ms / max(nface, 1)
    roofline = {"bound": "alu", "kernel": "k_single<Faces<D>> (face solve: prim->cons, fluxes, quartic speeds, HLLE)",
                "unit": "TFLOP/s", "peak": dfma_tflops,
                "peak_kind": "measured: FP64 FMA probe on this GPU (MEASURED_PEAKS.json has no FP64 entry)",
                "peak_nominal": nominal_tflops,
                "peak_nominal_kind": f"{sms} SMs (device) x {DFMA_PER_CLOCK_PER_SM} DFMA/clk x 2 flop x {max_mhz:.0f} MHz",
                "launch_ms": face_avg_ms, "launches": nface, "faces_per_launch": faces_per_launch,
                "flops_per_face": flops_per_face,
                "flops_per_face_literal": sf.get("face_solve_flops_per_face_literal"),
                "achieved": None, "frac": None, "traffic": read_traffic(args.n),
                "face_share_of_step": face_ms / ms if ms > 0 else None}
    if flops_per_face:
        achieved = flops_per_face * faces_per_launch / (face_avg_ms / 1e3) / 1e12
        roofline["achieved"] = achieved
        roofline["frac"] = achieved / dfma_tflops
    step_roofline = None
    if sf.get("flops_per_zone_stage"):
        fz = sf["flops_per_zone_stage"]
        ach = fz * value / world / 1e12
        step_roofline = {"bound": "alu", "unit": "TFLOP/s", "flops_per_zone_stage": fz,
                         "flops_per_zone_stage_literal_speed_iterations":
                             sf.get("flops_per_zone_stage_literal_speed_iterations"),
                         "achieved": ach, "peak": dfma_tflops, "frac": ach / dfma_tflops,
                         "bytes_per_zone_stage": 568, "hbm_gbs": 568 * value / world / 1e9}
    result = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
              "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
              "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
              "config": {"workload": WORKLOAD, "interior_cells": cells, "stages_per_step": 4,
                         "parallelism": f"replicas x{world}", "l2": "inputs larger than L2 (no flush)",
                         "resident_bytes": int(s.ws_bytes + 2 * U.numel() * 8 + P.numel() * 8 + M.numel() * 8),
                         "sm_count": sms},
              "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": io_bytes,
                      "d2h_bytes_per_step": io_bytes},
              "gpu_launches": LAUNCHES_PER_STAGE * 4 * args.steps,
              "clocks": clk, "roofline": roofline, "step_roofline": step_roofline,
              "c2p_counters_timed": {"n_noble": c2p[0], "n_fallback": c2p[1], "n_atm": c2p[2], "n_failed": c2p[3],
                                     "noble_iters": c2p[4]},
              "state_finite": finite}
    if not args.no_coupling:
        result["coupling"] = run_coupling(args, s, U, P, M, w, dev, stream)
    if not args.no_variants:
        result["variants"] = run_variants(args, s, U, P, w, dev, stream, U_warm, P_warm)
    del s, U, P, M, U_warm, P_warm
    torch.cuda.empty_cache()
    b128 = None if args.no_balsara else run_balsara(args, dev, stream)
    if b128:
        result["balsara_128"] = b128
    if not args.no_batched:
        result["batched"] = run_batched(args, dev, stream)
    if b128 and not args.no_tiled:
        result["tiled"] = run_tiled(args, dev, stream, b128["ms_per_step"])
    if b128 and not args.no_refined:
        result["refined"] = run_refined(args, dev, stream, b128["ms_per_step"])
    if not args.no_adjoint:
        result["adjoint"] = run_adjoint(args, dev, stream)
    if not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline(w)
    print(json.dumps(result))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)
    world, _, _ = dist_env()
    if world > 1:
        import torch.distributed as dist
        if dist.is_initialized():
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
