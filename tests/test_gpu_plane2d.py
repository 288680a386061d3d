"""The unconstrained 2D plane (surface kind xy2d, the baseline of the
performance comparison of Section 3.1) on the GPU against the oracle, both
precisions: interacting WCA particles move in the plane only, with the same
trajectory as the oracle's; the resident engine gives the same bits."""
import numpy as np
import pytest

from paper_1411_3019_gb300 import inputs as I
from paper_1411_3019_gb300 import md

from parity_util import POS_100, assert_forces, gpu_run, oracle_run

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_plane2d_matches_oracle(precision):
    _, plane = I.sphere_and_plane2d(n=800, seed=4, precision=precision,
                                    tol=1e-12 if precision == "fp64" else 1e-10)
    st, f, u, res, obs = gpu_run(plane, 80)
    ref, _, _, _, obs_ref = oracle_run(plane, 80)
    assert np.abs(st["x"] - ref["x"]).max() <= POS_100[precision]
    assert np.all(st["x"][:, 2] == plane[0]["x"][:, 2])
    assert np.all(st["v"][:, 2] == 0.0) and np.all(st["p_half"][:, 2] == 0.0)
    assert_forces(plane, st["x"], f, precision)
    assert obs[0]["ndof"] == 2 * plane[0]["n"]
    assert obs[0]["kT"] == pytest.approx(obs_ref[0]["kT"], rel=1e-6)


def test_plane2d_resident_bit_identical_and_sphere_counterpart_runs():
    sphere, plane = I.sphere_and_plane2d(n=1500, seed=5)
    runs = []
    for engine in (0, 1):
        sim = md.Simulation(plane)
        sim.set_state()
        if engine:
            md.md_set_option(sim.h, md.MD_OPT_ENGINE, 1)
        sim.step(30)
        sim.sync()
        runs.append(sim.state())
        sim.close()
    for key in ("x", "v", "p_half"):
        assert np.array_equal(runs[0][key], runs[1][key]), key
    st = gpu_run(sphere, 30)[0]
    assert np.abs(np.linalg.norm(st["x"], axis=1) - sphere[0]["surface"]["p"][0]).max() < 1e-8


def test_plane2d_rejects_a_periodic_z_axis():
    _, plane = I.sphere_and_plane2d(n=100, seed=6)
    plane[0]["params"] = dict(plane[0]["params"], periodic=(1, 1, 1), box_lo=(-20, -20, -20), box_hi=(20, 20, 20))
    with pytest.raises(md.MdError):
        md.Simulation(plane)
