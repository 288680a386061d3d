#!/usr/bin/env python
"""Throughput of the constrained Langevin time step (Algorithm S1 with
RATTLE, Algorithm 1) on one GB300, in particle-steps per second.

Workload (default `ellipsoid_torus`): 200,000 WCA particles at area
fraction 0.4 on an ellipsoid of shape (150, 120, 90) sigma scaled to
semi-axes (249.0, 199.2, 149.4) sigma, plus 50,000 on a torus R = 120,
r = 40 sigma as a separate system of the same batch; kT = gamma = 1,
dt = 0.002; float32 pair forces and noise, float64 state, constraint value,
projection and position update; RATTLE tolerance 1e-10 sigma. One bench
step = one time step of both systems (every kernel of the hot path).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl surfmd|reference]
                  [--workload NAME] [--precision mixed|fp64]

Prints one JSON line (rank 0). Under torchrun each rank advances its own,
independently seeded copy of the workload (weak scaling, no collective on
the data path; the timing uses a barrier and max/sum reductions only).
"""
from __future__ import annotations

import argparse
import datetime
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = ("particle-steps/sec on 1 GB300 (FP32-force/FP64-RATTLE vs plain FP64) at residual "
          "≤1e-10")
UNIT = "particle-steps/s"
L2_FLUSH_BYTES = 256 << 20  # larger than the 129 MB L2
WORKLOADS = ("ellipsoid_torus", "plain_sphere", "replicas", "bead_molecules", "bump_crowders", "nve_surfaces",
             "capsids", "sphere_vs_2d", "thylakoids", "lj_lattice")


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="surfmd", choices=["surfmd", "reference"])
    ap.add_argument("--workload", default="ellipsoid_torus", choices=WORKLOADS)
    ap.add_argument("--precision", default=None, choices=["mixed", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true", help="skip the float64 comparison leg")
    ap.add_argument("--no-tune", action="store_true",
                    help="keep the default launch options (with the Verlet list: the workload's skin and 32 "
                         "particles per warp, no autotuning)")
    ap.add_argument("--engine", default="auto", choices=["auto", "global", "resident"],
                    help="auto: the autotuner picks the engine and its options")
    ap.add_argument("--pair-tile", type=int, default=None, choices=[0, 8, 16, 32],
                    help="global engine with this cell-tiled pair kernel setting (0: per-particle rows) "
                         "instead of the autotuner's choice")
    ap.add_argument("--skin", type=float, default=-1.0,
                    help="> 0: Verlet neighbour list with this skin (cell edge r_c + skin), rebuilt when a "
                         "particle has moved skin / 2; 0: cell list every step; < 0: the workload's default")
    ap.add_argument("--max-neighbors", type=int, default=-1, help="< 0: the workload's default")
    ap.add_argument("--nrep", type=int, default=4096, help="systems of the replicas workload")
    ap.add_argument("--pair-form", type=int, default=1, choices=[0, 1],
                    help="nve_surfaces: 0 truncated-shifted, 1 linearly smoothed Lennard-Jones")
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    return ap.parse_args(argv)


# ---------------------------------------------------------------------------
# workloads and their sharding over ranks: the batched replicas are split
# across the ranks (strong scaling: the same 4,096 systems for any number of
# GPUs); every other workload is an independently seeded copy per rank (weak
# scaling)
# ---------------------------------------------------------------------------
def rank_seed(rank: int) -> int:
    return 1 + rank


def scaling_of(name: str) -> str:
    return "strong" if name == "replicas" else "weak"


def partition_replicas(systems, rank: int, world: int):
    """The replicas rank `rank` of `world` advances: largest first, each
    replica to the rank with the fewest particles so far (ties to the lowest
    rank), so every rank computes the same split; each keeps its systems in
    their original order (and with their own replica index and noise)."""
    load = [0] * world
    own = [[] for _ in range(world)]
    for k in sorted(range(len(systems)), key=lambda k: (-systems[k]["n"], k)):
        r = min(range(world), key=lambda q: (load[q], q))
        own[r].append(k)
        load[r] += systems[k]["n"]
    return [systems[k] for k in sorted(own[rank])]


def workload(name: str, rank: int, precision: str, nrep: int = 4096, pair_form: int = 1, world: int = 1):
    """The systems rank `rank` of `world` advances: its share of the batched
    replicas (the same batch on every rank, split by partition_replicas), or
    an independently seeded copy of any other workload."""
    from paper_1411_3019_gb300 import inputs

    seed = rank_seed(rank)
    if name == "replicas" and world > 1:
        full = inputs.c4_replicas(nrep=nrep, seed=rank_seed(0), precision=precision)
        return partition_replicas(full, rank, world)
    if name == "ellipsoid_torus":
        return inputs.c2_ellipsoid_torus(seed=seed, precision=precision)
    if name == "plain_sphere":
        return [inputs.sphere_system(1000, 10.0, seed=seed, dmin=0.8, precision=precision, dt=0.001,
                                     tol=1e-12 if precision == "fp64" else 1e-10)]
    if name == "replicas":
        return inputs.c4_replicas(nrep=nrep, seed=seed, precision=precision)
    if name == "bead_molecules":
        return inputs.c5_bead_molecules(seed=seed, precision=precision)
    if name == "bump_crowders":
        return inputs.c3_bump_crowders(seed=seed, precision=precision)
    if name == "sphere_vs_2d":
        return inputs.sphere_and_plane2d(n=250_000, seed=seed, precision=precision)[0]
    if name == "thylakoids":  # 128 crowded thylakoids of the SI (2500 crowders, bridge radius 1.5)
        out = []
        for k in range(max(1, nrep // 32)):
            sy = inputs.thylakoid_system(n=2500, Rb=1.5, seed=seed * 100_003 + k, precision=precision,
                                         dmin=0.9)[0]
            sy["params"] = dict(sy["params"], replica=k)
            out.append(sy)
        return out
    if name == "capsids":
        return inputs.capsid_systems(nsys=max(1, nrep // 4), ncone=60, seed=seed, precision=precision)
    if name == "nve_surfaces":
        return inputs.nve_systems(pair_form, seed=seed, precision=precision,
                                  tol=1e-12 if precision == "fp64" else 1e-10)
    if name == "lj_lattice":  # dense free LJ liquid, 97,336 particles, rc = 2.5 (pair-kernel stress case)
        return inputs.lj_lattice(46, seed=seed + 2, precision=precision,
                                 tol=1e-12 if precision == "fp64" else 1e-10)
    raise ValueError(name)


# Verlet list (skin, entries per particle) per workload when --skin is not
# given. On every workload measured the list on the global engine is faster
# than a cell list every step (1.7-2.2x) and than the resident engine's
# batches (replicas 5.8e9 vs 4.6e9, capsids 1.5e9 vs 1.3e9, thylakoids 1.4e9
# vs 1.1e9 particle-steps/s); --skin 0 restores the per-step cell list (and
# with it the autotuner's engine choice). The NVE study keeps the cell list.
DEFAULT_NLIST = {"ellipsoid_torus": (0.4, 64), "bump_crowders": (0.4, 64), "bead_molecules": (0.4, 128),
                 "sphere_vs_2d": (0.5, 64), "lj_lattice": (0.3, 128), "replicas": (0.4, 64),
                 "capsids": (0.4, 256), "thylakoids": (0.4, 64), "plain_sphere": (0.4, 64)}


def workload_skin(args) -> float:
    if args.skin >= 0:
        return args.skin
    # the resident engine keeps its own per-step cell lists
    return 0.0 if args.engine == "resident" else DEFAULT_NLIST.get(args.workload, (0.0, 0))[0]


def workload_max_neighbors(args) -> int:
    return DEFAULT_NLIST.get(args.workload, (0.0, 64))[1] if args.max_neighbors < 0 else args.max_neighbors


def cells_for_skin(systems, skin: float):
    """With a neighbour list the cell edge must be at least r_c + skin."""
    if skin > 0:
        for sy in systems:
            sy["params"] = dict(sy["params"], cell_size=float(max(map(max, sy["params"]["rcut"]))) + skin)
    return systems


def workload_config(name, systems, precision):
    n = int(sum(s["n"] for s in systems))
    if name == "ellipsoid_torus":
        ell, tor = systems[0]["surface"]["p"], systems[1]["surface"]["p"]
        desc = (f"ellipsoid+torus: {systems[0]['n']} WCA on ellipsoid semi-axes "
                f"({ell[0]:.1f},{ell[1]:.1f},{ell[2]:.1f}) at phi=0.4 + {systems[1]['n']} on torus "
                f"R={tor[0]:g} r={tor[1]:g} (separate system); kT=gamma=1, dt=0.002, tol=1e-10")
    elif name == "sphere_vs_2d":
        desc = (f"sphere_vs_2d: {n} WCA on a sphere R={systems[0]['surface']['p'][0]:.1f} at phi=0.4 (RATTLE), "
                f"against the same n in a periodic 2D plane at the same density (unconstrained_2d)")
    elif name == "nve_surfaces":
        desc = (f"nve_surfaces: {len(systems)} x {systems[0]['n']} LJ (rc=2.5) on "
                f"{'/'.join(s['name'] for s in systems)} at phi=0.3, gamma=0, dt=0.0005, "
                f"pair_form={systems[0]['params'].get('pair_form', 0)}")
    else:
        desc = f"{name}: {n} particles in {len(systems)} system(s)"
    return {"workload": f"{desc}, {precision}", "particles": n, "systems": len(systems),
            "precision": precision,
            "l2": "flushed between timed steps (256 MB written, then read back so no line is dirty; outside the "
                  "timed events)"}


def reduce_over_ranks(dist, ms_local: float, n_local: float, device=None):
    """(max over ranks of the step time, total particles over ranks)."""
    if dist is None:
        return ms_local, n_local
    import torch

    t = torch.tensor([ms_local], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    m = torch.tensor([n_local], dtype=torch.float64, device=device)
    dist.all_reduce(m, op=dist.ReduceOp.SUM)
    return float(t.item()), float(m.item())


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi sampling every 50 ms from construction to stop(); only the
    samples whose timestamps fall inside [mark_start, mark_end] are kept."""
    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.proc = None
        self.t0 = self.t1 = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50", "-i", str(device_index)], stdout=self.file, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def mark_start(self):
        self.t0 = datetime.datetime.now()

    def mark_end(self):
        self.t1 = datetime.datetime.now()

    @staticmethod
    def parse(text: str, t0, t1):
        sm, smax, reasons, n_all = [], [], set(), 0
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in text.splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f")
                mhz, mhz_max = float(parts[2]), float(parts[3])
            except ValueError:
                continue
            n_all += 1
            if t0 is not None and not (t0 <= ts <= t1):
                continue
            sm.append(mhz)
            smax.append(mhz_max)
            for nm, val in zip(names, parts[6:10]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm), "window_s": round((t1 - t0).total_seconds(), 3) if t0 else None}

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        text = self.file.read()
        os.unlink(self.file.name)
        return self.parse(text, self.t0, self.t1)


# ---------------------------------------------------------------------------
# rooflines
# ---------------------------------------------------------------------------
# Algorithmic bytes per particle of the two kernels every step runs (each
# datum the method needs read or written once):
#   integrate: x (24) + p^{k-1/2} (24) + f (12, float32; 24 on the float64
#              path) + type/flags (4) read, x + p^{k-1/2} (48) written, the
#              cell key (4)  -> 116 B (128 B float64 path)
#   pair:      the particle's float4 record once (16; double4 32), its cell
#              start (4) and the force written (16; 32)  -> 36 B (68 B float64)
ALGO_BYTES = {"mixed": {"integrate": 116, "pair": 36}, "fp64": {"integrate": 128, "pair": 68}}


def algorithmic_bytes(kernel: str, n: int, nbucket: int, precision: str, nlist: bool = False) -> float:
    """Algorithmic bytes of one launch: the per-particle figure above times
    the particles for the integrator and the pair kernel (either step form);
    for the cell-list kernels (cell list every step) the bytes they move if
    every datum is read or written once; the list build and, with the
    neighbour list, the cell-list kernels (rebuild steps only) count none."""
    if kernel in ("integrate", "pair"):
        return float(ALGO_BYTES[precision][kernel] * n)
    if nlist:
        return 0.0
    v4 = 16 if precision == "mixed" else 32
    tiles = math.ceil(nbucket / 8192)
    per = {
        # counters read and cleared, starts written, tile states
        "scan": 12 * nbucket + 16 * tiles,
        # cell id, rank, bucket start; slot written
        "scatter": n * (4 + 4 + 4 + 4),
        # slot id, cell, meta, x (3 x float64), bucket range; record, sorted id, sorted cell
        "bucket_build": n * (4 + 4 + 4 + 24 + 8 + v4 + 4 + 4),
        # resident engine, per step: meta, x, p_half read; x, p_half written (the
        # cell list and forces stay in shared memory)
        "resident": n * (4 + 24 + 24 + 24 + 24),
    }
    return float(per.get(kernel, 0))


def impl_bytes(kernel: str, n: int, precision: str, nlist: bool) -> float:
    """Bytes the implementation's launch reads and writes once each (beyond
    the algorithmic count: the list step's slot map, build position and the
    records it moves; the float4 force's energy word)."""
    v4 = 16 if precision == "mixed" else 32
    lo = 16 if precision == "mixed" else 0
    if kernel == "integrate":
        base = 4 + 24 + 24 + v4 + 24 + 24
        return float(n * (base + (4 + 24 + v4 + lo + v4 + lo if nlist else 4 + 4)))
    if kernel == "pair":
        return float(n * (4 + 4 + v4 + lo + 4 + v4))
    return 0.0


def kernels_source_hash() -> str:
    path = os.path.join(ROOT, "paper_1411_3019_gb300", "csrc", "kernels.cu")
    with open(path, "rb") as fh:
        return hashlib.sha256(fh.read()).hexdigest()


def ncu_counts(workload_name: str, precision: str, nlist: bool = False):
    """Per-launch ncu counters (float64-pipe thread instructions, DRAM bytes)
    recorded in profiles/ for this workload (and step form: neighbour list or
    cell list every step), if they were taken from the current kernel source
    (else {})."""
    suffix = "_nlist" if nlist else ""
    path = os.path.join(ROOT, "profiles", f"ncu_counts_{workload_name}_{precision}{suffix}.txt")
    if not os.path.exists(path):
        return {}
    out, sha = {}, None
    with open(path) as fh:
        for line in fh:
            parts = line.split()
            if not parts or parts[0].startswith("#"):
                continue
            if parts[0] == "kernels_cu_sha256":
                sha = parts[1]
            elif len(parts) == 3:
                out.setdefault(parts[0], {})[parts[1]] = float(parts[2])
    return out if sha == kernels_source_hash() else {}


def rooflines(prof_ms, n, nbucket, precision, hbm_peak, counts, fma_peaks, nlist=False):
    """Per-kernel achieved bandwidth against the measured HBM copy peak, and
    the float64 / float32 pipe fractions where ncu counts of the current
    kernel source are recorded (instructions per launch / duration / the FMA
    instruction rate measured in this run). The headline roofline is the
    dominant (longest) kernel's HBM fraction on its algorithmic bytes."""
    table = {}
    for k, ms in prof_ms.items():
        b = algorithmic_bytes(k, n, nbucket, precision, nlist)
        row = {"ms": round(ms, 5), "bytes_per_launch": b, "hbm_gbs": b / (ms / 1e3) / 1e9,
               "hbm_frac": b / (ms / 1e3) / 1e9 / hbm_peak}
        ib = impl_bytes(k, n, precision, nlist)
        if ib:
            row["impl_bytes_per_launch"] = ib
        c = counts.get(k, {})
        if "fp64_inst" in c and fma_peaks.get("fp64"):
            row["fp64_inst_per_launch"] = c["fp64_inst"]
            row["fp64_pipe_frac"] = c["fp64_inst"] / (ms / 1e3) / fma_peaks["fp64"]
        if "dram_bytes" in c:
            row["traffic"] = c["dram_bytes"]
        if "fma_pct" in c:  # sm__pipe_fma_cycles_active: the float32 pipe's busy fraction (ncu)
            row["fp32_pipe_frac"] = c["fma_pct"] / 100.0
        table[k] = row
    top = max(prof_ms, key=prof_ms.get)
    r = table[top]
    main = {"bound": "hbm", "kernel": top, "achieved": r["hbm_gbs"], "peak": hbm_peak, "unit": "GB/s",
            "frac": r["hbm_frac"], "traffic": r.get("traffic"),
            "bytes_per_unit": ALGO_BYTES[precision].get(top), "units_per_launch": n,
            "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs, copy)"}
    for key in ("fp64_pipe_frac", "fp32_pipe_frac"):
        if key in r:
            main[key] = r[key]
    main["per_kernel"] = table
    return main


# ---------------------------------------------------------------------------
# the GPU arm
# ---------------------------------------------------------------------------
def main(argv=None):
    args = parse(argv)
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    precision = args.precision or ("fp64" if args.workload in ("plain_sphere", "nve_surfaces") else "mixed")
    if args.impl == "reference":
        return reference_arm(args, rank, world, precision)

    import torch

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_1411_3019_gb300 import md

    def barrier():
        if dist is not None:
            dist.barrier()

    stream = torch.cuda.Stream()
    clocks = ClockSampler(local) if rank == 0 else None  # sampling from here; the timed window is marked below
    flush_buf = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    flush_out = torch.empty((), dtype=torch.float32, device="cuda")

    def flush_l2():
        """Write a buffer larger than L2, then read it back, so that the L2
        holds none of the workload's data and none of its lines are dirty
        (the next kernel does not pay for the flush's write-back)."""
        flush_buf.add_(1.0)
        torch.amax(flush_buf, dim=0, out=flush_out)

    def timed_steps(sim, k):
        """k steps, each bracketed by CUDA events on the launching stream; the
        L2 is flushed between steps outside the events."""
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(k)]
        launches = 0
        with torch.cuda.stream(stream):
            for a, b in evs:
                flush_l2()
                a.record(stream)
                sim.step(1)
                launches += md.md_last_launch_count(sim.h)
                b.record(stream)
        stream.synchronize()
        return [a.elapsed_time(b) for a, b in evs], launches

    def timed_resident(sim, k):
        """k steps in one md_step call (the resident engine's persistent
        launches plus its one cell-list rebuild), bracketed by CUDA events;
        the L2 is flushed before; the state (x and p) is larger than L2."""
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            flush_l2()
            a.record(stream)
            sim.step(k)
            b.record(stream)
        stream.synchronize()
        return [a.elapsed_time(b) / k] * k, md.md_last_launch_count(sim.h)

    skin = workload_skin(args)
    systems = workload(args.workload, rank, precision, args.nrep, args.pair_form, world)
    list_tuned = None
    if skin > 0 and args.skin < 0 and not args.no_tune and args.engine != "resident":
        from paper_1411_3019_gb300 import tune

        with torch.cuda.stream(stream):  # the skin (cell size r_c + skin) and the walk's warp width
            list_tuned = tune.autotune_list(systems, workload_max_neighbors(args), flush=lambda: flush_l2(),
                                            stream=stream)
        if list_tuned:
            skin = list_tuned["skin"]
    systems = cells_for_skin(systems, skin)
    n_local = int(sum(s["n"] for s in systems))
    sim = md.Simulation(systems, stream=stream)
    if skin > 0:
        md.md_set_neighbor_list(sim.h, skin, workload_max_neighbors(args))
        if list_tuned:
            md.md_set_option(sim.h, md.MD_OPT_LIST_WARP, list_tuned["list_warp"])
    sim.set_state()
    sim.step(args.warmup)
    sim.sync()
    from paper_1411_3019_gb300 import tune

    tuned = {"options": {"pair_order": md.md_get_option(sim.h, md.MD_OPT_PAIR_ORDER),
                         "pair_lanes": md.md_get_option(sim.h, md.MD_OPT_PAIR_LANES)}}
    if args.engine == "resident":
        md.md_set_option(sim.h, md.MD_OPT_ENGINE, 1)
        tuned = {"options": {"engine": 1, "resident_threads": md.md_get_option(sim.h, md.MD_OPT_RESIDENT_THREADS)}}
    elif skin > 0:
        tuned = {"options": {"neighbor_list_skin": skin, "max_neighbors": workload_max_neighbors(args)},
                 "trials": list_tuned["trials"] if list_tuned else None}
        if precision != "fp64":
            tuned["options"]["list_warp"] = md.md_get_option(sim.h, md.MD_OPT_LIST_WARP)
    elif args.pair_tile is not None:
        md.md_set_option(sim.h, md.MD_OPT_PAIR_TILE, args.pair_tile)
        tuned = {"options": {**tuned["options"], "pair_tile": args.pair_tile}}
    elif args.engine == "auto" and not args.no_tune:
        with torch.cuda.stream(stream):  # launch options chosen by the autotuner during warm-up
            tuned = tune.autotune(sim.h, trials=3, flush=lambda: flush_l2())
    sim.step(2)
    sim.sync()
    builds0 = md.md_get_option(sim.h, md.MD_OPT_NLIST_BUILDS) if skin > 0 else 0

    barrier()
    torch.cuda.synchronize()
    if clocks:
        clocks.mark_start()
    t_wall0 = time.perf_counter()
    resident = md.md_get_option(sim.h, md.MD_OPT_ENGINE) == 1
    durs, launches = (timed_resident if resident else timed_steps)(sim, args.steps)
    if skin > 0:  # list builds in the timed steps (the rebuild kernels exit at once in the others)
        tuned["options"]["rebuilds_in_timed_steps"] = md.md_get_option(sim.h, md.MD_OPT_NLIST_BUILDS) - builds0
    torch.cuda.synchronize()
    barrier()
    t_wall = time.perf_counter() - t_wall0
    if clocks:
        clocks.mark_end()
    clk = clocks.stop() if clocks else None
    sim.sync()
    res = sim.residual()
    ms, total_particles = reduce_over_ranks(dist, sum(durs) / len(durs), float(n_local), "cuda")
    value = total_particles / (ms / 1e3)

    # steady state: back-to-back steps without flushes (state resident in L2)
    with torch.cuda.stream(stream):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        sim.step(args.steps)
        b.record(stream)
    stream.synchronize()
    ms_resident, _ = reduce_over_ranks(dist, a.elapsed_time(b) / args.steps, 0.0, "cuda")

    # per-kernel durations (events between kernels, L2 flushed between steps)
    prof = {}
    nprof = min(args.steps, 20)
    with torch.cuda.stream(stream):
        if resident:  # the resident launches per step and the rebuild of one call spread over its steps
            flush_l2()
            prof = md.md_profile_step(sim.h, min(args.steps, 100))
        else:
            for _ in range(nprof):
                flush_l2()
                for kname, kms in md.md_profile_step(sim.h, 1).items():
                    prof[kname] = prof.get(kname, 0.0) + kms / nprof
    nbucket = int(md.md_cell_list(sim.h)["bucket_start"].shape[0] - 1)
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            peaks = json.load(fh)
    except OSError:
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    fma_peaks = {"fp64": md.md_measure_fma_peak("fp64"), "fp32": md.md_measure_fma_peak("mixed")}
    roofline = rooflines(prof, n_local, nbucket, precision, hbm_peak, ncu_counts(args.workload, precision, skin > 0),
                         fma_peaks, nlist=skin > 0)
    roofline["fma_peaks_measured"] = {"fp64_fma_per_s": fma_peaks["fp64"], "fp32_fma_per_s": fma_peaks["fp32"]}
    if "hbm_gbs" not in peaks:
        roofline["peak_source"] = "fallback (6.8 TB/s)"

    # end to end through the C ABI with host buffers (pinned): restore the
    # checkpoint state from the host, one step, read the state back
    st = sim.state()
    hx = torch.empty((n_local, 3), dtype=torch.float64, pin_memory=True).numpy()
    hp = torch.empty((n_local, 3), dtype=torch.float64, pin_memory=True).numpy()
    hx[:] = st["x"]
    hp[:] = st["p_half"]
    k_now = st["step"]
    import ctypes as C
    L = md.lib()
    xp, pp = hx.ctypes.data_as(C.c_void_p), hp.ctypes.data_as(C.c_void_p)
    step_c = C.c_uint64()
    e2e_n = max(1, args.e2e_steps)
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_n):
        rc = L.md_restore(sim.h, xp, pp, k_now)
        rc |= L.md_step(sim.h, 1)
        rc |= L.md_get_state(sim.h, xp, None, pp, C.byref(step_c))
        if rc:
            raise RuntimeError(md.md_last_error(sim.h))
        k_now = step_c.value
    e2e_s, _ = reduce_over_ranks(dist, (time.perf_counter() - t0) / e2e_n, 0.0, "cuda")
    e2e = {"value": total_particles / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 2 * 24 * n_local,
           "d2h_bytes_per_step": 2 * 24 * n_local + 8, "ms_per_step": e2e_s * 1e3,
           "path": "md_restore(host x, p_half) + md_step(1) + md_get_state(host x, p_half)"}
    # the state the accuracy report starts from (the benched launch configuration), and one more step
    snap = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not resident:
        s_k = sim.state()
        f_k, _ = sim.forces()
        sim.step(1)
        sim.sync()
        snap = {"state": s_k, "forces": f_k, "next": sim.state()}
    sim.close()
    diffusion = diffusion_check(md, stream) if precision == "mixed" and rank == 0 else None

    plain = None
    if not args.no_plain and precision == "mixed":
        systems64 = cells_for_skin(workload(args.workload, rank, "fp64", args.nrep, args.pair_form, world), skin)
        sim64 = md.Simulation(systems64, stream=stream)
        if skin > 0:
            md.md_set_neighbor_list(sim64.h, skin, workload_max_neighbors(args))
        sim64.set_state()
        sim64.step(args.warmup)
        sim64.sync()
        k64 = max(10, args.steps // 4)
        barrier()
        d64, _ = timed_steps(sim64, k64)
        sim64.sync()
        res64 = sim64.residual()
        ms64, _ = reduce_over_ranks(dist, sum(d64) / len(d64), 0.0, "cuda")
        plain = {"value": total_particles / (ms64 / 1e3), "unit": UNIT, "ms_per_step": ms64, "steps": k64,
                 "dtype": "f64", "max_g_over_gradg": res64["max_g_over_gradg"],
                 "mixed_speedup": ms64 / ms}
        sim64.close()

    # the performance comparison of Section 3.1: the same number of particles
    # at the same density in a periodic 2D plane with no constraint
    flat = None
    if args.workload == "sphere_vs_2d":
        from paper_1411_3019_gb300 import inputs

        plane = cells_for_skin(inputs.sphere_and_plane2d(n=250_000, seed=rank_seed(rank), precision=precision)[1],
                               skin)
        simp = md.Simulation(plane, stream=stream)
        if skin > 0:
            md.md_set_neighbor_list(simp.h, skin, workload_max_neighbors(args))
        simp.set_state()
        simp.step(args.warmup)
        simp.sync()
        if args.engine == "auto" and not args.no_tune and skin <= 0:
            with torch.cuda.stream(stream):
                tune.autotune(simp.h, trials=3, flush=lambda: flush_l2())
        barrier()
        dp, _ = timed_steps(simp, args.steps)
        simp.close()
        msp, _ = reduce_over_ranks(dist, sum(dp) / len(dp), 0.0, "cuda")
        flat = {"value": total_particles / (msp / 1e3), "unit": UNIT, "ms_per_step": msp,
                "workload": "250000 WCA in a periodic 2D plane (z updates not evaluated) at the sphere's "
                            "area fraction 0.4", "rattle_over_2d": ms / msp}

    cpu, accuracy = None, {"residual_max_g_over_gradg": res["max_g_over_gradg"], "diffusion": diffusion}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu, acc = oracle_leg(systems, args.cpu_seconds, snap, precision)
        accuracy.update(acc)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": scaling_of(args.workload),
            "vs_baseline": None, "dtype": "f32+f64" if precision == "mixed" else "f64", "data": "synthetic",
            "config": dict(workload_config(args.workload, systems, precision),
                           **({"l2": f"one md_step({args.steps}) call (persistent resident launches), L2 flushed "
                                     f"before it; the state x, p ({48 * n_local / 1e6:.0f} MB) is larger than "
                                     f"the 129 MB L2"} if resident else {}),
                           engine="resident" if resident else "global"),
            "residual_max_g_over_gradg": res["max_g_over_gradg"],
            "l2_resident": {"value": total_particles / (ms_resident / 1e3), "ms_per_step": ms_resident},
            "wall_s_timed_region": t_wall,
            "roofline": roofline, "cpu_baseline": cpu, "accuracy": accuracy, "e2e": e2e, "clocks": clk,
            "gpu_launches": launches, "plain_fp64": plain, "unconstrained_2d": flat,
            "tuned": {"options": tuned["options"], "trials": tuned.get("trials")},
        }
        if scaling_of(args.workload) == "strong" and world > 1:  # the whole batch, split over the ranks
            line["config"].update(particles=int(total_particles), systems=args.nrep,
                                  workload=f"replicas: {int(total_particles)} particles in {args.nrep} systems, "
                                           f"split across {world} ranks by particle count, {precision}")
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def _oracle_systems(systems):
    import oracle

    sims = []
    for s in systems:
        o = oracle.System(s["surface"], s["params"], s["n"], force_mode="cells")
        o.set_state(s["x"], s["v"], s["type"], s.get("mol"), s["constrained"])
        sims.append(o)
    return sims


def cpu_info() -> dict:
    """Host cores and CPU model (lscpu, else /proc/cpuinfo)."""
    cores = os.cpu_count() or 1
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if model is None:
        try:
            with open("/proc/cpuinfo") as fh:
                for line in fh:
                    if line.lower().startswith(("model name", "cpu part")):
                        model = line.split(":", 1)[1].strip()
                        break
        except OSError:
            pass
    return {"cores": cores, "model": model}


def time_oracle(systems, seconds: float, threads: int):
    """Whole time steps of the oracle on `threads` host threads for about
    `seconds`; returns (particle-steps/s, steps, elapsed, threads used)."""
    import oracle

    used = oracle.set_threads(threads)
    sims = _oracle_systems(systems)
    n = sum(s["n"] for s in systems)
    steps = 0
    t0 = time.perf_counter()
    while True:
        for o in sims:
            o.step(1)
        steps += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    oracle.set_threads(1)
    return n * steps / el, steps, el, used


def oracle_leg(systems, seconds: float, snap, precision: str):
    """The oracle on the host cores (the CPU baseline: single-threaded and
    with OpenMP over the particle loops on every core, whole time steps of the
    same workload, about `seconds` each) and the accuracy of the GPU run
    against it: forces of every particle at the benched state, and one step of
    Algorithm S1 (position half with its multiplier) for sampled particles."""
    import oracle

    info = cpu_info()
    n = sum(s["n"] for s in systems)
    v1, k1, e1, _ = time_oracle(systems, seconds, 1)
    vm, km, em, used = time_oracle(systems, seconds, info["cores"])
    cpu = {"value": vm, "unit": UNIT, "cores": used, "kind": "oracle", "model": info["model"],
           "sample": f"{km} whole time steps of the {n}-particle workload ({len(systems)} system(s)), {em:.1f} s, "
                     f"float64 C oracle with a cell list, OpenMP over the per-particle loops on {used} threads",
           "single_thread": {"value": v1, "cores": 1, "sample": f"{k1} whole time steps, {e1:.1f} s"}}
    acc = {}
    if snap is not None:
        acc.update(force_accuracy(systems, snap))
        acc.update(step_accuracy(systems, snap))
    return cpu, acc


def _oracle_forces(systems, x):
    import oracle

    out, off = [], 0
    for s in systems:
        xs = x[off:off + s["n"]]
        mol = s.get("mol")
        if mol is None:
            bpm = s["params"].get("beads_per_mol", 0)
            mol = (np.arange(s["n"]) // bpm if bpm > 1 else np.arange(s["n"])).astype(np.int32)
        f, _ = oracle.pair_forces(s["params"], xs, s["type"], mol, mode="cells")
        fb, _, _ = oracle.bond_wall_forces(s["params"], xs, s["constrained"], s["type"])
        out.append(f + fb)
        off += s["n"]
    return np.concatenate(out)


def force_accuracy(systems, snap):
    """|df| / max(|f|, 1 eps/sigma) of every particle's force at the benched state."""
    x, f = snap["state"]["x"], snap["forces"]
    ref = _oracle_forces(systems, x)
    rel = np.linalg.norm(f - ref, axis=1) / np.maximum(np.linalg.norm(ref, axis=1), 1.0)
    return {"force_rel_err": {"max": float(rel.max()), "p99_99": float(np.quantile(rel, 0.9999)),
                              "above_1e-5": int((rel > 1e-5).sum()), "particles": int(rel.size),
                              "metric": "|f_gpu - f_oracle| / max(|f_oracle|, 1 eps/sigma), all particles",
                              "step": int(snap["state"]["step"])}}


def step_accuracy(systems, snap, per_system: int = 200):
    """One step of Algorithm S1 from the GPU's state for sampled constrained
    particles (the oracle advances each with its neighbours at the GPU's
    positions): the largest |x^{k+1}_gpu - x^{k+1}_oracle| and the multiplier
    difference it implies, as the normal constraint force |dlambda n0| =
    |dx . n0| / (a |n0|) with a = dt^2 / (2m) (eps/sigma)."""
    import oracle

    st, nxt = snap["state"], snap["next"]
    k = int(st["step"])
    g = np.random.default_rng(7)
    dx_max, dlam_max, count = 0.0, 0.0, 0
    off = 0
    for s in systems:
        sl = slice(off, off + s["n"])
        off += s["n"]
        x, ph, xn = st["x"][sl], st["p_half"][sl], nxt["x"][sl]
        con = np.nonzero(s["constrained"])[0]
        if con.size == 0:
            continue
        m = s["params"]["mass"][0]
        a = s["params"]["dt"] ** 2 / (2 * m)
        for i in g.choice(con, size=min(per_system, con.size), replace=False):
            _, xa, _, _ = oracle.particle_advance(s["surface"], s["params"], x, int(i), ph[i], k, 0, s["type"],
                                                   None, s["constrained"])
            _, n0 = oracle.surface_g(s["surface"], s["params"], x[i])
            d = xn[i] - xa
            dx_max = max(dx_max, float(np.abs(d).max()))
            dlam_max = max(dlam_max, abs(float(d @ n0)) / (a * float(np.linalg.norm(n0))))
            count += 1
    return {"position_half": {"max_abs_dx": dx_max, "max_abs_dlambda_n0": dlam_max, "particles": count,
                              "step": k,
                              "metric": "one step of Algorithm S1 from the GPU's (x^k, p^{k-1/2}) per sampled "
                                        "constrained particle; |dlambda n0| = |dx . n0| / (a |n0|), "
                                        "a = dt^2/(2m), in eps/sigma"}}


def diffusion_check(md, stream):
    """Diffusion coefficient of 40,000 non-interacting particles on a sphere of
    radius 10 (mixed path, same library): <r(0).r(t)>/R^2 = exp(-2 D t'/R^2),
    t' = t - tau(1 - e^{-t/tau}) (SI S1.3 with the Langevin inertia; tau = 1),
    fitted through the origin in ln c over t = 10, 25, 50, 80; D = kT/(m gamma) = 1."""
    from paper_1411_3019_gb300 import inputs

    R, dt = 10.0, 0.002
    surf = {"kind": "sphere", "center": (0.0, 0.0, 0.0), "p": (R, 0.0, 0.0, 0.0)}
    sim = md.Simulation(inputs.free_on_surface(surf, 40_000, seed=3, dt=dt), stream=stream)
    sim.set_state()
    ts, cs, t = [], [], 0.0
    for tc in (10.0, 25.0, 50.0, 80.0):
        k = int(round((tc - t) / dt))
        sim.step(k)
        t += k * dt
        ts.append(t - (1 - math.exp(-t)))
        cs.append(sim.observables()[0]["r0_dot_rt"])
    sim.close()
    ts, lc = np.array(ts), np.log(np.array(cs))
    d_fit = float(-(ts @ lc) / (ts @ ts) * R ** 2 / 2)
    return {"D_fit": d_fit, "D_theory": 1.0, "rel_err": d_fit - 1.0,
            "setup": "40000 non-interacting particles on a sphere R=10, mixed, dt=0.002, t up to 80 tau"}


def reference_arm(args, rank: int, world: int, precision: str):
    """The reference arm is the oracle on the host cores (OpenMP over its
    per-particle loops on every core): rank 0 only, whole time steps of the
    same workload (at most 60 timed steps)."""
    if rank != 0:
        return
    import oracle

    info = cpu_info()
    threads = oracle.set_threads(info["cores"])
    systems = workload(args.workload, 0, precision, args.nrep, args.pair_form)
    sims = _oracle_systems(systems)
    n = sum(s["n"] for s in systems)
    for _ in range(args.warmup):
        for o in sims:
            o.step(1)
    steps = max(1, min(args.steps, 60))
    t0 = time.perf_counter()
    for _ in range(steps):
        for o in sims:
            o.step(1)
    el = time.perf_counter() - t0
    value = n * steps / el
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": steps,
            "warmup": args.warmup, "ms_per_step": el / steps * 1e3, "higher_is_better": True,
            "scaling": scaling_of(args.workload), "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(workload_config(args.workload, systems, precision),
                           engine="resident" if args.engine == "resident" else "global"),
            "impl": "reference",
            "cpu_baseline": {"kind": "oracle", "cores": threads, "model": info["model"], "value": value,
                             "unit": UNIT,
                             "sample": f"{steps} whole time steps of the {n}-particle workload, OpenMP over the "
                                       f"per-particle loops on {threads} threads"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
