"""Failure paths, made on the host: bad states, an iteration cap that the
Newton solve cannot meet, a particle that leaves its grid, a non-finite
momentum. Each comes back as a status code and the context stays usable."""
import numpy as np
import pytest

from paper_1411_3019_gb300 import inputs as I
from paper_1411_3019_gb300 import md

pytestmark = pytest.mark.gpu


def _sphere(**kw):
    return I.sphere_system(n=200, R=6.0, seed=2, dmin=0.9, precision="mixed", **kw)


def _healthy():
    s = _sphere()
    with md.Simulation([s]) as sim:
        sim.set_state()
        sim.step(5)
        sim.sync()
        assert sim.residual()["max_g_over_gradg"] < 1e-10


def test_off_surface_state_is_rejected():
    s = _sphere()
    s["x"] = s["x"].copy()
    s["x"][3] *= 1.01
    with md.Simulation([s]) as sim:
        with pytest.raises(md.MdError) as e:
            sim.set_state()
        assert e.value.code == md.MD_ERR_INVALID_ARG
        with pytest.raises(md.MdError):  # no valid state: stepping is refused
            sim.step(1)
    _healthy()


def test_type_outside_ntypes_is_rejected():
    """A particle type equal to ntypes (inside the table's 8 slots, outside
    the types the parameters define) is refused by md_set_state."""
    s = _sphere()
    s["type"] = np.asarray(s["type"]).copy()
    s["type"][5] = s["params"]["ntypes"]
    with md.Simulation([s]) as sim:
        with pytest.raises(md.MdError) as e:
            sim.set_state()
        assert e.value.code == md.MD_ERR_INVALID_ARG
    _healthy()


def test_nan_state_is_rejected():
    s = _sphere()
    s["v"] = s["v"].copy()
    s["v"][0, 0] = np.nan
    with md.Simulation([s]) as sim, pytest.raises(md.MdError) as e:
        sim.set_state()
    assert e.value.code == md.MD_ERR_INVALID_ARG
    _healthy()


def test_newton_cap_reports_rattle_divergence():
    s = _sphere()
    s["params"] = dict(s["params"], max_newton=0, rattle_tol=1e-14)
    with md.Simulation([s]) as sim:
        sim.set_state()
        sim.step(2)
        with pytest.raises(md.MdError) as e:
            sim.sync()
        assert e.value.code == md.MD_ERR_RATTLE_DIVERGED
        sim.sync()  # the status word was cleared when reported
    _healthy()


def test_particle_leaving_the_grid_is_reported():
    prm = I.wca_params(box_lo=(-5, -5, -5), box_hi=(5, 5, 5), gamma=0.0, kT=0.0)
    x = np.array([[0.0, 0.0, 0.0], [3.0, 3.0, 3.0]])
    v = np.array([[50.0, 0.0, 0.0], [0.0, 0.0, 0.0]])
    s = I._system("free", {"kind": "none"}, prm, x, v)
    with md.Simulation([s]) as sim:
        sim.set_state()
        sim.step(100)
        assert md.md_status(sim.h) & md.MD_FLAG_OUT_OF_GRID
    _healthy()


def test_non_finite_momentum_is_reported():
    prm = I.wca_params(box_lo=(-5, -5, -5), box_hi=(5, 5, 5))
    x = np.array([[0.0, 0.0, 0.0], [3.0, 3.0, 3.0]])
    s = I._system("free", {"kind": "none"}, prm, x, np.zeros((2, 3)))
    with md.Simulation([s]) as sim:
        sim.set_state()
        sim.step(1)
        st = sim.state()
        ph = st["p_half"].copy()
        ph[0, 1] = np.inf
        md.md_restore(sim.h, st["x"], ph, st["step"])
        sim.step(1)
        flags = md.md_status(sim.h)
        assert flags & md.MD_FLAG_NONFINITE
    _healthy()


def test_empty_and_single_particle_systems():
    s0 = _sphere()
    s0.update(n=0, x=np.zeros((0, 3)), v=np.zeros((0, 3)), type=np.zeros(0, np.int32),
              constrained=np.zeros(0, np.uint8))
    with md.Simulation([s0]) as sim:
        sim.set_state()
        sim.step(3)
        sim.sync()
        assert sim.state()["x"].shape == (0, 3)
        assert md.md_info(sim.h)["step"] == 3
    s1 = _sphere()
    s1.update(n=1, x=s1["x"][:1], v=s1["v"][:1], type=s1["type"][:1], constrained=s1["constrained"][:1])
    with md.Simulation([s1]) as sim:
        sim.set_state()
        sim.step(10)
        sim.sync()
        f, _ = sim.forces()
        assert np.abs(f).max() == 0.0
        assert sim.residual()["max_g_over_gradg"] < 1e-10


def test_scan_wait_limit_reports_timeout_and_the_next_step_recovers():
    """The scan's bounded look-back wait (the one device-side wait): with a
    limit of 0 reads every tile after the first gives up, latches the
    timeout flag and returns (no wait, every access in bounds); the next
    synchronising call reports MD_ERR_TIMEOUT, and the next md_step rebuilds
    the cell list, so the run then repeats a run that never timed out bit
    for bit."""
    systems = I.c2_ellipsoid_torus(n_ell=4000, n_tor=1500, seed=8, precision="mixed")
    with md.Simulation(systems) as ref:
        ref.set_state()
        ref.step(4)
        ref.sync()
        want = ref.state()
    with md.Simulation(systems) as sim:
        sim.set_state()
        assert md.md_get_option(sim.h, md.MD_OPT_SPIN_LIMIT) == 1 << 22
        assert md.md_cell_list(sim.h)["bucket_start"].shape[0] - 1 > 8192  # more than one scan tile
        md.md_set_option(sim.h, md.MD_OPT_SPIN_LIMIT, 0)
        sim.step(1)
        with pytest.raises(md.MdError) as e:
            sim.sync()
        assert e.value.code == md.MD_ERR_TIMEOUT
        sim.sync()  # reported once, then cleared
        md.md_set_option(sim.h, md.MD_OPT_SPIN_LIMIT, 1 << 22)
        sim.step(3)
        sim.sync()
        got = sim.state()
        assert sim.residual()["max_g_over_gradg"] < 1e-10
    assert got["step"] == want["step"] == 4
    for key in ("x", "p_half"):
        assert np.array_equal(got[key], want[key]), key
    with md.Simulation(systems) as sim, pytest.raises(md.MdError):
        md.md_set_option(sim.h, md.MD_OPT_SPIN_LIMIT, -1)
