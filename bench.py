#!/usr/bin/env python
"""Throughput of the constrained Langevin time step (Algorithm S1 with
RATTLE, Algorithm 1) on one GB300, in particle-steps per second.

Workload (default): 200,000 WCA particles at area fraction 0.4 on an
ellipsoid of shape (150, 120, 90) sigma scaled to semi-axes
(249.0, 199.2, 149.4) sigma, plus 50,000 on a torus R = 120, r = 40 sigma as a
separate system of the same batch; kT = gamma = 1, dt = 0.002; float32 pair
forces and noise, float64 state, Newton solve, projection and position
update; RATTLE tolerance 1e-10 sigma. One bench step = one time step of
both systems (every kernel of the hot path).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl surfmd|reference]

Prints one JSON line (rank 0). Under torchrun each rank advances its own,
independently seeded copy of the workload (weak scaling, no collective on
the data path).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = ("particle-steps/sec on 1 GB300 (FP32-force/FP64-RATTLE vs plain FP64) at residual "
          "≤1e-10")
UNIT = "particle-steps/s"
L2_FLUSH_BYTES = 256 << 20  # larger than the 129 MB L2


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="surfmd", choices=["surfmd", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true", help="skip the float64 comparison leg")
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    return ap.parse_args()


def workload(rank: int, precision: str = "mixed"):
    from paper_1411_3019_gb300 import inputs

    systems = inputs.c2_ellipsoid_torus(seed=1 + rank, precision=precision)
    return systems


def workload_config(systems, precision):
    ell, tor = systems[0]["surface"]["p"], systems[1]["surface"]["p"]
    return {
        "workload": (f"ellipsoid+torus: {systems[0]['n']} WCA on ellipsoid semi-axes "
                     f"({ell[0]:.1f},{ell[1]:.1f},{ell[2]:.1f}) at phi=0.4 + {systems[1]['n']} on torus "
                     f"R={tor[0]:g} r={tor[1]:g} (separate system); kT=gamma=1, dt=0.002, "
                     f"tol=1e-10, {precision}"),
        "particles": int(sum(s["n"] for s in systems)),
        "systems": len(systems),
        "precision": precision,
        "l2": "flushed between timed steps (256 MB write, outside the timed events)",
    }


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(device_index)], stdout=self.file, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

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
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.file.read().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.file.name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# algorithmic bytes per launch of each kernel
# ---------------------------------------------------------------------------
def algorithmic_bytes(kernel: str, n: int, nbucket: int, precision: str) -> float:
    v4 = 16 if precision == "mixed" else 32
    per = {
        # fused: pair reads (sorted id, cell, own record, meta) + update reads x, p and writes
        # x, p, cell, rank (+ bucket starts once, counters read-modify-write)
        "pair_integrate": n * (4 + 4 + v4 + 4 + 24 + 24 + 24 + 24 + 4 + 4) + 4 * (nbucket + 1) + 8 * nbucket,
        # reads: sorted id, cell id, own record, meta; write: force vec4 (+ bucket starts once)
        "pair": n * (4 + 4 + v4 + 4 + v4) + 4 * (nbucket + 1),
        # reads: meta, x, p_half, force vec4; writes: x, p_half, cell, rank; counter RMW
        "integrate": n * (4 + 24 + 24 + v4 + 24 + 24 + 4 + 4) + 8 * nbucket,
        # counters read and cleared, starts written, chunk sums read
        "scan": 12 * nbucket + 4 * math.ceil(nbucket / 4096),
        # cell id and rank read, bucket start read, slot written
        "scatter": n * (4 + 4 + 4 + 4),
        "bucket_build": n * (4 + 4 + 4 + 24 + 4 + v4) + 4 * (nbucket + 1) + 4 * n,
    }
    return float(per.get(kernel, 0))


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return reference_arm(args, rank, world)

    import numpy as np
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

    def max_over_ranks(v: float) -> float:
        if dist is None:
            return v
        t = torch.tensor([v], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    def sum_over_ranks(v: float) -> float:
        if dist is None:
            return v
        t = torch.tensor([v], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        return float(t.item())

    stream = torch.cuda.Stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def timed_steps(sim, k):
        """k steps, each bracketed by CUDA events on the launching stream; the
        L2 is flushed between steps outside the events."""
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(k)]
        launches = 0
        with torch.cuda.stream(stream):
            for a, b in evs:
                flush.add_(1.0)
                a.record(stream)
                sim.step(1)
                launches += md.md_last_launch_count(sim.h)
                b.record(stream)
        stream.synchronize()
        return [a.elapsed_time(b) for a, b in evs], launches

    precision = "mixed"
    systems = workload(rank, precision)
    n_local = int(sum(s["n"] for s in systems))
    sim = md.Simulation(systems, stream=stream)
    sim.set_state()
    sim.step(args.warmup)
    sim.sync()

    barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local) if rank == 0 else None
    t_wall0 = time.perf_counter()
    durs, launches = timed_steps(sim, args.steps)
    torch.cuda.synchronize()
    barrier()
    t_wall = time.perf_counter() - t_wall0
    clk = clocks.stop() if clocks else None
    sim.sync()
    res = sim.residual()
    ms_local = sum(durs) / len(durs)
    ms = max_over_ranks(ms_local)
    total_particles = sum_over_ranks(float(n_local))
    value = total_particles / (ms / 1e3)

    # steady state: back-to-back steps without flushes (state resident in L2)
    with torch.cuda.stream(stream):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        sim.step(args.steps)
        b.record(stream)
    stream.synchronize()
    ms_resident = max_over_ranks(a.elapsed_time(b) / args.steps)

    # per-kernel durations (events between kernels, L2 flushed between steps)
    prof = {}
    nprof = min(args.steps, 20)
    with torch.cuda.stream(stream):
        for _ in range(nprof):
            flush.add_(1.0)
            for kname, kms in md.md_profile_step(sim.h, 1).items():
                prof[kname] = prof.get(kname, 0.0) + kms / nprof
    nbucket = int(md.md_cell_list(sim.h)["bucket_start"].shape[0] - 1)
    top = max(prof, key=prof.get)
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            peaks = json.load(fh)
    except OSError:
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    achieved = algorithmic_bytes(top, n_local, nbucket, precision) / (prof[top] / 1e3) / 1e9
    roofline = {"bound": "hbm", "kernel": top, "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak, "traffic": None,
                "peak_source": "measured" if "hbm_gbs" in peaks else "fallback",
                "kernel_ms": {k: round(v, 5) for k, v in prof.items()},
                "bytes_per_launch": algorithmic_bytes(top, n_local, nbucket, precision)}

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
    e2e_s = max_over_ranks((time.perf_counter() - t0) / e2e_n)
    e2e = {"value": total_particles / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 2 * 24 * n_local,
           "d2h_bytes_per_step": 2 * 24 * n_local + 8, "ms_per_step": e2e_s * 1e3,
           "path": "md_restore(host x, p_half) + md_step(1) + md_get_state(host x, p_half)"}
    sim.close()

    plain = None
    if not args.no_plain:
        systems64 = workload(rank, "fp64")
        sim64 = md.Simulation(systems64, stream=stream)
        sim64.set_state()
        sim64.step(args.warmup)
        sim64.sync()
        k64 = max(10, args.steps // 4)
        barrier()
        d64, _ = timed_steps(sim64, k64)
        sim64.sync()
        res64 = sim64.residual()
        ms64 = max_over_ranks(sum(d64) / len(d64))
        plain = {"value": total_particles / (ms64 / 1e3), "unit": UNIT, "ms_per_step": ms64, "steps": k64,
                 "dtype": "f64", "max_g_over_gradg": res64["max_g_over_gradg"],
                 "mixed_speedup": ms64 / ms}
        sim64.close()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(workload(0, precision), args.cpu_seconds)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": workload_config(systems, precision),
            "residual_max_g_over_gradg": res["max_g_over_gradg"],
            "l2_resident": {"value": total_particles / (ms_resident / 1e3), "ms_per_step": ms_resident},
            "wall_s_timed_region": t_wall,
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk,
            "gpu_launches": launches, "plain_fp64": plain,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def cpu_baseline(systems, seconds: float):
    """The oracle, as it stands, on the host cores: whole time steps of the same
    workload for about `seconds` of CPU time (single thread)."""
    import oracle

    sims = []
    for s in systems:
        o = oracle.System(s["surface"], s["params"], s["n"], force_mode="cells")
        o.set_state(s["x"], s["v"])
        sims.append(o)
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
    return {"value": n * steps / el, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{steps} whole time steps of the {n}-particle workload (both systems), "
                      f"{el:.1f} s, single-threaded float64 C oracle with a cell list"}


def reference_arm(args, rank: int, world: int):
    """The reference arm is the oracle on the host cores: rank 0 only."""
    if rank != 0:
        return
    import oracle

    systems = workload(0, "mixed")
    sims = []
    for s in systems:
        o = oracle.System(s["surface"], s["params"], s["n"], force_mode="cells")
        o.set_state(s["x"], s["v"])
        sims.append(o)
    n = sum(s["n"] for s in systems)
    for _ in range(args.warmup):
        for o in sims:
            o.step(1)
    steps = min(args.steps, 60)
    t0 = time.perf_counter()
    for _ in range(steps):
        for o in sims:
            o.step(1)
    el = time.perf_counter() - t0
    value = n * steps / el
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": steps,
            "warmup": args.warmup, "ms_per_step": el / steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(systems, "mixed"), "impl": "reference",
            "cpu_baseline": {"kind": "oracle", "cores": 1, "value": value, "unit": UNIT,
                             "sample": f"{steps} whole time steps of the {n}-particle workload"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
