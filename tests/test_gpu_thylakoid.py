"""The thylakoid composite surface of SI S3.1 on the GPU: crowded WCA
particles against the oracle on the same seeded input in both precisions
(pieces chosen where each half step starts and held for the solve, so both
sides cross the junctions the same way), free particles diffusing over the
junctions, and the resident engine against the global one."""
import numpy as np
import pytest

from paper_1411_3019_gb300 import inputs as I
from paper_1411_3019_gb300 import md

from parity_util import POS_100, assert_forces, gpu_run, oracle_run

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("Rb", [1.5, 2.5])
def test_thylakoid_matches_oracle(precision, Rb):
    systems = I.thylakoid_system(n=2000, Rb=Rb, seed=7, precision=precision,
                                 tol=1e-12 if precision == "fp64" else 1e-10)
    st, f, u, res, _ = gpu_run(systems, 60)
    ref = oracle_run(systems, 60)[0]
    assert np.abs(st["x"] - ref["x"]).max() <= POS_100[precision]
    assert_forces(systems, st["x"], f, precision)
    # residual measured on the piece at the end position: second order near junctions
    assert res["max_g_over_gradg"] < 1e-5


def test_free_particles_cross_the_junctions():
    systems = I.thylakoid_system(n=3000, seed=8, interacting=False)
    sim = md.Simulation(systems)
    sim.set_state()
    x0 = systems[0]["x"]
    on_bridge0 = np.abs(x0[:, 0]) < 5.0
    sim.step(20000)
    sim.sync()
    st = sim.state()
    res = sim.residual()
    sim.close()
    assert res["max_g_over_gradg"] < 1e-5
    # particles have moved between the blocks and the bridge in both directions
    on_bridge1 = np.abs(st["x"][:, 0]) < 5.0
    assert np.sum(on_bridge0 & ~on_bridge1) > 0 and np.sum(~on_bridge0 & on_bridge1) > 0


def test_thylakoid_resident_engine_bit_identical():
    systems = I.thylakoid_system(n=1500, seed=9)
    runs = []
    for engine in (0, 1):
        sim = md.Simulation(systems)
        sim.set_state()
        if engine:
            md.md_set_option(sim.h, md.MD_OPT_ENGINE, 1)
        sim.step(40)
        sim.sync()
        runs.append(sim.state())
        sim.close()
    for key in ("x", "v", "p_half"):
        assert np.array_equal(runs[0][key], runs[1][key]), key
