"""Energy conservation at gamma = 0, after the energy-conservation study of
the SI: 500 Lennard-Jones particles (cutoff 2.5 sigma) held on a sphere, a
cylinder, a torus and a plane, dt = 0.0005, float64. The total energy
H = K + U must stay within a small fraction of its start value, and the
linearly smoothed potential (force continuous at the cutoff) must conserve it
clearly better than the truncated-shifted one (force jump at the cutoff),
the qualitative result the SI reports."""
import numpy as np
import pytest

from paper_1411_3019_gb300 import inputs as I
from paper_1411_3019_gb300 import md

pytestmark = pytest.mark.gpu

STEPS, EVERY = 100_000, 5_000


def _max_rel_dev(form):
    systems = I.nve_systems(form)
    sim = md.Simulation(systems)
    sim.set_state()
    H = []
    for k in range(STEPS // EVERY + 1):
        if k:
            sim.step(EVERY)
        H.append([o["kinetic"] + o["potential"] for o in sim.observables()])
    res = sim.residual()
    sim.close()
    H = np.array(H)
    assert res["max_g_over_gradg"] < 1e-12
    return {s["name"]: float(np.abs(H[:, j] - H[0, j]).max() / abs(H[0, j])) for j, s in enumerate(systems)}


def test_linearly_smoothed_lj_conserves_energy_better_than_truncated():
    trunc = _max_rel_dev(0)
    smooth = _max_rel_dev(1)
    for name in smooth:
        assert smooth[name] < 2e-5, (name, smooth[name])
        assert trunc[name] < 1e-3, (name, trunc[name])
    assert np.mean(list(trunc.values())) > 2.0 * np.mean(list(smooth.values())), (trunc, smooth)
