"""Launch options of the step (visiting order and lanes per particle of the
pair kernel) and the autotuner that picks them: every setting gives forces
and trajectories within the parity tolerances of the oracle, and the visiting
order, which only permutes which thread handles which particle, changes no
bit of the trajectory."""
import numpy as np
import pytest

from paper_1411_3019_gb300 import inputs as I
from paper_1411_3019_gb300 import md, tune

from parity_util import POS_100, assert_forces, oracle_run

pytestmark = pytest.mark.gpu


def _systems(precision):
    tol = 1e-12 if precision == "fp64" else 1e-10
    return I.c4_replicas(nrep=3, seed=8, nmin=200, nmax=600, rmin=6.0, rmax=10.0, precision=precision,
                         dt=0.002, tol=tol)


def _run(systems, nsteps, opts=None):
    opts = opts or {}
    sim = md.Simulation(systems)
    for key, val in opts.items():
        md.md_set_option(sim.h, key, val)
    sim.set_state()
    sim.step(nsteps)
    sim.sync()
    got = {k: md.md_get_option(sim.h, k) for k in opts}
    st = sim.state()
    f, _ = sim.forces()
    sim.close()
    return st, f, got


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("lanes", [1, 2, 4, 8])
@pytest.mark.parametrize("order", [0, 1])
def test_every_option_setting_matches_oracle(precision, lanes, order):
    systems = _systems(precision)
    st, f, got = _run(systems, 30, {md.MD_OPT_PAIR_LANES: lanes, md.MD_OPT_PAIR_ORDER: order})
    assert got == {md.MD_OPT_PAIR_LANES: lanes, md.MD_OPT_PAIR_ORDER: order}
    ref = oracle_run(systems, 30)[0]
    assert np.abs(st["x"] - ref["x"]).max() <= POS_100[precision]
    assert_forces(systems, st["x"], f, precision)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_visiting_order_changes_no_bit(precision):
    systems = _systems(precision)
    a = _run(systems, 40, {md.MD_OPT_PAIR_ORDER: 0})
    b = _run(systems, 40, {md.MD_OPT_PAIR_ORDER: 1})
    for key in ("x", "v", "p_half"):
        assert np.array_equal(a[0][key], b[0][key]), key
    assert np.array_equal(a[1], b[1])


def test_switching_options_mid_run_keeps_the_trajectory():
    systems = _systems("mixed")
    ref = _run(systems, 48)[0]
    sim = md.Simulation(systems)
    sim.set_state()
    for order in (0, 1, 0):
        md.md_set_option(sim.h, md.MD_OPT_PAIR_ORDER, order)
        sim.step(16)
    sim.sync()
    st = sim.state()
    sim.close()
    for key in ("x", "v", "p_half"):
        assert np.array_equal(st[key], ref[key]), key


def test_bad_option_values_are_rejected():
    sim = md.Simulation(_systems("mixed"))
    for key, val in ((md.MD_OPT_PAIR_LANES, 3), (md.MD_OPT_PAIR_ORDER, 2), (md.MD_OPT_PAIR_TILE, 1), (md.MD_OPT_PAIR_TILE, 2), (99, 1)):
        with pytest.raises(md.MdError):
            md.md_set_option(sim.h, key, val)
    sim.close()


def test_autotuner_applies_a_valid_choice_and_keeps_parity(tmp_path):
    systems = _systems("mixed")
    sim = md.Simulation(systems)
    sim.set_state()
    cache = str(tmp_path / "tune.json")
    out = tune.autotune(sim.h, trials=1, cache=cache)
    # six global settings (visiting order x lanes), the cell-tiled pair kernel
    # at three run lengths (these small grids have cell-id buckets) and three
    # resident CTA sizes
    assert len(out["trials"]) == 12 and out["trials"][0]["ms"] == out["best_ms"]
    assert sorted(t["engine"] for t in out["trials"]) == [0] * 9 + [1] * 3
    assert sorted(t.get("pair_tile", 0) for t in out["trials"] if t.get("pair_tile")) == [8, 16, 32]
    opts = out["options"]
    assert md.md_get_option(sim.h, md.MD_OPT_ENGINE) == opts["engine"]
    if opts["engine"] == 0 and opts["pair_tile"]:
        assert md.md_get_option(sim.h, md.MD_OPT_PAIR_TILE) == opts["pair_tile"]
    elif opts["engine"] == 0:
        assert opts["pair_order"] in (0, 1) and opts["pair_lanes"] in (1, 2, 4)
        assert md.md_get_option(sim.h, md.MD_OPT_PAIR_ORDER) == opts["pair_order"]
        assert md.md_get_option(sim.h, md.MD_OPT_PAIR_TILE) == 0
    else:
        assert md.md_get_option(sim.h, md.MD_OPT_RESIDENT_THREADS) == opts["resident_threads"]
    again = tune.autotune(sim.h, cache=cache)
    assert again["cached"] and again["options"] == out["options"]
    # the trial steps advanced the state: restart from the inputs and compare
    sim.set_state()
    sim.step(30)
    sim.sync()
    st = sim.state()
    f, _ = sim.forces()
    sim.close()
    ref = oracle_run(systems, 30)[0]
    assert np.abs(st["x"] - ref["x"]).max() <= POS_100["mixed"]
    assert_forces(systems, st["x"], f, "mixed")


def test_list_autotuner_times_every_skin_and_warp_width():
    """tune.autotune_list creates one handle per skin (cell edge r_c + skin),
    times each particles-per-warp setting over steps that include its list
    rebuilds, and returns the fastest; a handle with the chosen setting then
    matches the oracle."""
    systems = I.c2_ellipsoid_torus(n_ell=4000, n_tor=1500, seed=8, precision="mixed")
    out = tune.autotune_list(systems, 128, skins=(0.2, 0.4), list_warps=(32, 16), steps=30, warmup=5)
    assert out is not None and len(out["trials"]) == 4
    assert {(t["skin"], t["list_warp"]) for t in out["trials"]} == {(0.2, 32), (0.2, 16), (0.4, 32), (0.4, 16)}
    assert out["trials"][0]["ms"] == out["best_ms"] and all(t["builds"] >= 0 for t in out["trials"])
    assert all("cell_size" not in s["params"] or s["params"]["cell_size"] == 0.0 for s in systems)  # inputs untouched
    chosen = tune._with_cell_size(systems, out["skin"])
    with md.Simulation(chosen) as sim:
        md.md_set_neighbor_list(sim.h, out["skin"], 128)
        md.md_set_option(sim.h, md.MD_OPT_LIST_WARP, out["list_warp"])
        sim.set_state()
        sim.step(20)
        sim.sync()
        x = sim.state()["x"]
    ref = oracle_run(systems, 20)[0]
    assert np.abs(x - ref["x"]).max() <= POS_100["mixed"]
