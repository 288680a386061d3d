"""The capsid model of SI S3.2 (cones of four beads with type-dependent bond
lengths, bend angles, one bead held on a sphere, a spherical wall, mixed
bead sizes and attraction between like beads) on the GPU against the oracle
on the same seeded input, in both precisions, and the resident engine
against the global one."""
import numpy as np
import pytest

from paper_1411_3019_gb300 import inputs as I
from paper_1411_3019_gb300 import md

from parity_util import POS_100, assert_forces, gpu_run, oracle_run

pytestmark = pytest.mark.gpu


def _capsids(precision, nsys=2, ncone=40):
    return I.capsid_systems(nsys=nsys, ncone=ncone, seed=3, precision=precision,
                            tol=1e-12 if precision == "fp64" else 1e-10)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_capsid_forces_and_trajectory_match_oracle(precision):
    systems = _capsids(precision)
    st0, f0, u0, _, _ = gpu_run(systems, 0)
    assert_forces(systems, st0["x"], f0, precision)
    st, f, u, res, _ = gpu_run(systems, 60)
    ref, _, u_ref, _, _ = oracle_run(systems, 60)
    assert np.abs(st["x"] - ref["x"]).max() <= POS_100[precision]
    assert_forces(systems, st["x"], f, precision)
    np.testing.assert_allclose(u.sum(), u_ref.sum(), rtol=1e-9 if precision == "fp64" else 1e-5)
    assert res["max_g_over_gradg"] < systems[0]["params"]["rattle_tol"]


def test_bent_cones_feel_the_bend_potential():
    systems = _capsids("fp64", nsys=1, ncone=20)
    sy = systems[0]
    g = np.random.default_rng(4)
    x = sy["x"].copy()
    free = sy["constrained"] == 0
    x[free] += g.normal(0, 0.08, (free.sum(), 3))  # bend every cone a little
    sy["x"] = x
    _, f, u, _, _ = gpu_run(systems, 0)
    _, f_ref, u_ref, _, _ = oracle_run(systems, 0)
    np.testing.assert_allclose(f, f_ref, rtol=1e-10, atol=1e-9)
    np.testing.assert_allclose(u.sum(), u_ref.sum(), rtol=1e-12)


def test_capsid_resident_engine_bit_identical():
    systems = _capsids("mixed", nsys=4)
    runs = []
    for engine in (0, 1):
        sim = md.Simulation(systems)
        sim.set_state()
        if engine:
            md.md_set_option(sim.h, md.MD_OPT_ENGINE, 1)
        sim.step(25)
        sim.sync()
        runs.append((sim.state(), sim.forces()))
        sim.close()
    for key in ("x", "v", "p_half"):
        assert np.array_equal(runs[0][0][key], runs[1][0][key]), key
    assert np.array_equal(runs[0][1][0], runs[1][1][0])
