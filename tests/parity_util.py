"""Shared helpers of the GPU parity tests: run a list of system dicts on the
GPU (through the C ABI) and on the oracle (one oracle system per system),
and compare."""
from __future__ import annotations

import numpy as np

import oracle
from paper_1411_3019_gb300 import md

# Tolerances of the float64 path and of the mixed path.
# Forces: fp64 is checked as |df| / max(|f|, 1); mixed (float32 pair
# arithmetic) as |df| / max(S, 1) with S the particle's force scale, the sum
# of the magnitudes of its pair/bond/wall terms (the net force can cancel).
FORCE_REL = {"fp64": 1e-11, "mixed": 1e-5}
POS_100 = {"fp64": 1e-8, "mixed": 1e-6}


def force_err(f_gpu, f_ref):
    """max |df| / max(|f|, 1) per particle (1 eps/sigma floor for near-zero forces)."""
    scale = np.maximum(np.linalg.norm(f_ref, axis=1), 1.0)
    return float(np.max(np.linalg.norm(f_gpu - f_ref, axis=1) / scale)) if len(f_ref) else 0.0


def gpu_run(systems, nsteps, step0=0, chunks=None, opts=None):
    sim = md.Simulation(systems)
    for key, val in (opts or {}).items():
        md.md_set_option(sim.h, key, val)
        assert md.md_get_option(sim.h, key) == val
    sim.set_state(step0)
    for k in (chunks or [nsteps]):
        if k:
            sim.step(k)
    sim.sync()
    st = sim.state()
    f, u = sim.forces()
    res = sim.residual()
    obs = sim.observables()
    sim.close()
    return st, f, u, res, obs


def oracle_run(systems, nsteps, step0=0, force_mode="auto"):
    xs, vs, phs, fs, us, res, obs = [], [], [], [], [], [], []
    for s in systems:
        o = oracle.System(s["surface"], s["params"], s["n"], force_mode=force_mode)
        o.set_state(s["x"], s["v"], s["type"], s.get("mol"), s["constrained"], step0)
        o.step(nsteps)
        st = o.state()
        f, u = o.forces()
        xs.append(st["x"])
        vs.append(st["v"])
        phs.append(st["p_half"])
        fs.append(f)
        us.append(u)
        res.append(o.residual())
        obs.append(o.observables())
    cat = np.concatenate
    return {"x": cat(xs), "v": cat(vs), "p_half": cat(phs)}, cat(fs), cat(us), res, obs


def oracle_force_scale_at(systems, x):
    out, off = [], 0
    for s in systems:
        xs = x[off:off + s["n"]]
        out.append(oracle.force_scale(s["params"], xs, s["type"], s.get("mol"), s["constrained"],
                                      s["surface"]))
        off += s["n"]
    return np.concatenate(out) if out else np.zeros(0)


def assert_forces(systems, x, f_gpu, precision):
    """GPU forces at x against the oracle at the same x; returns the measured
    errors (net-relative and scale-relative)."""
    f_ref = oracle_forces_at(systems, x)
    d = np.linalg.norm(f_gpu - f_ref, axis=1)
    net_rel = float(np.max(d / np.maximum(np.linalg.norm(f_ref, axis=1), 1.0))) if len(d) else 0.0
    if precision == "fp64":
        assert net_rel <= FORCE_REL["fp64"], net_rel
        return net_rel, net_rel
    scale = oracle_force_scale_at(systems, x)
    scale_rel = float(np.max(d / np.maximum(scale, 1.0))) if len(d) else 0.0
    assert scale_rel <= FORCE_REL["mixed"], (scale_rel, net_rel)
    return net_rel, scale_rel


def oracle_forces_at(systems, x):
    """Oracle forces (pair + bond + wall) of every system at the positions x
    (all systems concatenated) -- isolates the force kernel from trajectory
    differences."""
    out, off = [], 0
    for s in systems:
        xs = x[off:off + s["n"]]
        mol = s.get("mol")
        if mol is None:
            bpm = s["params"].get("beads_per_mol", 0)
            mol = (np.arange(s["n"]) // bpm if bpm > 1 else np.arange(s["n"])).astype(np.int32)
        f, _ = oracle.pair_forces(s["params"], xs, s["type"], mol)
        fb, _, _ = oracle.bond_wall_forces(s["params"], xs, s["constrained"], s["type"])
        out.append(f + fb)
        off += s["n"]
    return np.concatenate(out) if out else np.zeros((0, 3))


def precision_of(systems):
    p = systems[0]["params"]["precision"]
    return p if isinstance(p, str) else ("fp64" if p == 0 else "mixed")
