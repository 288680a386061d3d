"""Shared helpers of the GPU parity tests: run a list of system dicts on the
GPU (through the C ABI) and on the oracle (one oracle system per system),
and compare."""
from __future__ import annotations

import numpy as np

import oracle
from paper_1411_3019_gb300 import md

# Tolerances of the float64 path and of the mixed path.
# Forces: both precisions are checked per particle as |df| / max(|f|, 1 eps/sigma)
# (the per-particle relative error with a floor for near-zero forces). The
# mixed path's error is also reported relative to the particle's force scale
# S (the sum of the magnitudes of its pair, bond and wall terms), which shows
# how much of it comes from cancellation in the net force.
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


# Pairs the oracle may evaluate all-against-all per call of oracle_forces_at;
# above, its forces use its cell list (which its pins check against all pairs).
BRUTE_PAIRS = 4e8


def _brute(systems):
    return sum(float(s["n"]) ** 2 for s in systems) <= BRUTE_PAIRS


def force_errors(systems, x, f_gpu):
    """Per-particle |df| / max(|f|, 1) and |df| / max(S, 1) of GPU forces at x
    against the oracle at the same x (S, the force scale, is computed by the
    oracle over all pairs, so only where that is affordable; NaN otherwise)."""
    f_ref = oracle_forces_at(systems, x)
    d = np.linalg.norm(np.asarray(f_gpu) - f_ref, axis=1)
    net = d / np.maximum(np.linalg.norm(f_ref, axis=1), 1.0)
    if _brute(systems):
        sc = d / np.maximum(oracle_force_scale_at(systems, x), 1.0)
    else:
        sc = np.full(len(d), np.nan)
    return net, sc


def assert_forces(systems, x, f_gpu, precision):
    """GPU forces at x against the oracle at the same x, held to
    |df| / max(|f|, 1) <= FORCE_REL[precision] on every particle; returns
    the largest net-relative and scale-relative errors."""
    net, sc = force_errors(systems, x, f_gpu)
    net_rel = float(net.max()) if len(net) else 0.0
    scale_rel = float(np.max(sc)) if len(sc) else 0.0
    assert net_rel <= FORCE_REL[precision], (net_rel, scale_rel)
    return net_rel, scale_rel


def oracle_forces_at(systems, x):
    """Oracle forces (pair + bond + wall) of every system at the positions x
    (all systems concatenated) -- isolates the force kernel from trajectory
    differences."""
    out, off = [], 0
    mode = "brute" if _brute(systems) else "cells"
    for s in systems:
        xs = x[off:off + s["n"]]
        mol = s.get("mol")
        if mol is None:
            bpm = s["params"].get("beads_per_mol", 0)
            mol = (np.arange(s["n"]) // bpm if bpm > 1 else np.arange(s["n"])).astype(np.int32)
        f, _ = oracle.pair_forces(s["params"], xs, s["type"], mol, mode=mode)
        fb, _, _ = oracle.bond_wall_forces(s["params"], xs, s["constrained"], s["type"])
        out.append(f + fb)
        off += s["n"]
    return np.concatenate(out) if out else np.zeros((0, 3))


def precision_of(systems):
    p = systems[0]["params"]["precision"]
    return p if isinstance(p, str) else ("fp64" if p == 0 else "mixed")
