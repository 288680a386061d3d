"""Full-size workloads in the configuration the benchmark times, checked on
sampled particles that the oracle computes one by one: the force on each
sampled particle (all pairs with it), the first step after the state is set
and a later step (Algorithm S1 for that particle, its neighbours at the
GPU's positions), plus the constraint residual of every particle."""
import numpy as np
import pytest

import oracle
from paper_1411_3019_gb300 import inputs as I
from paper_1411_3019_gb300 import md

from parity_util import FORCE_REL

pytestmark = pytest.mark.gpu

_cache = {}


def _workload(name):
    if name not in _cache:
        if name == "ellipsoid_torus_250k":
            _cache[name] = I.c2_ellipsoid_torus()
        elif name == "replicas_4096":
            _cache[name] = I.c4_replicas()
    return _cache[name]


def _sample(n, k, seed):
    g = np.random.default_rng(seed)
    return np.unique(np.concatenate([[0, n - 1], g.choice(n, size=min(k, n), replace=False)]))


def _check_system(sy, x0, f0, x1, ph1, x2, sample_k, seed, dx_tol):
    prm, surf = sy["params"], sy["surface"]
    idx = _sample(sy["n"], sample_k, seed)
    small = sy["n"] <= 5000
    scale_all = oracle.force_scale(prm, x0, sy["type"], None, sy["constrained"], surf) if small else None
    for i in idx:
        f_ref, _ = oracle.force_on(prm, x0, i, sy["type"], None, sy["constrained"], surf)
        sc = scale_all[i] if small else _scale_on(prm, x0, i, sy)
        assert np.linalg.norm(f0[i] - f_ref) / max(sc, 1.0) <= FORCE_REL["mixed"]
        m = prm["mass"][sy["type"][i]]
        _, xa, pha, st = oracle.particle_advance(surf, prm, x0, i, sy_p0(sy, i), 0, 1, sy["type"], None,
                                                 sy["constrained"])
        assert st >= 0
        assert np.abs(xa - x1[i]).max() <= dx_tol
        _, xb, _, st = oracle.particle_advance(surf, prm, x1, i, ph1[i], 1, 0, sy["type"], None,
                                               sy["constrained"])
        assert st >= 0
        assert np.abs(xb - x2[i]).max() <= dx_tol
        del m


def _scale_on(prm, x, i, sy):
    """Force scale of particle i alone: its neighbours within the largest cutoff
    (a superset of its interacting pairs) as a small system."""
    rc = float(np.max(prm["rcut"]))
    near = np.nonzero(np.sum((x - x[i]) ** 2, axis=1) < (rc + 1e-9) ** 2)[0]
    j = int(np.nonzero(near == i)[0][0])
    return oracle.force_scale(prm, x[near], sy["type"][near], None, sy["constrained"][near],
                              sy["surface"])[j]


def sy_p0(sy, i):
    """p^0 of particle i as md_set_state stores it: m v projected on the
    tangent plane (the projection is the oracle's, at x^0)."""
    x, v = sy["x"][i], sy["v"][i]
    m = sy["params"]["mass"][sy["type"][i]]
    if sy["constrained"][i]:
        _, n = oracle.surface_g(sy["surface"], sy["params"], x)
        v = v - (n @ v) / (n @ n) * n
    return m * v


@pytest.mark.parametrize("name,sample_k", [("ellipsoid_torus_250k", 150), ("replicas_4096", 40)])
def test_full_size_sampled_parity(name, sample_k):
    systems = _workload(name)
    with md.Simulation(systems) as sim:
        sim.set_state()
        f0, _ = sim.forces()
        sim.step(1)
        sim.sync()
        s1 = sim.state()
        sim.step(1)
        sim.sync()
        s2 = sim.state()
        res = sim.residual()
    assert res["max_g_over_gradg"] <= 1e-10
    off = 0
    picks = range(len(systems)) if len(systems) <= 2 else np.linspace(0, len(systems) - 1, 5).astype(int)
    offs = np.concatenate([[0], np.cumsum([s["n"] for s in systems])])
    for k in picks:
        sy = systems[k]
        off = offs[k]
        sl = slice(off, off + sy["n"])
        _check_system(sy, sy["x"], f0[sl], s1["x"][sl], s1["p_half"][sl], s2["x"][sl], sample_k,
                      seed=int(k), dx_tol=1e-9)
