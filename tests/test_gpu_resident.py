"""The resident engine (one persistent launch, one CTA per system with its
cell list and forces in shared memory) against the global engine: the same
per-particle code in the same order, so every bit of the trajectory must
agree; plus the oracle, the launch options, switching engines mid-run and
the systems the engine must refuse."""
import numpy as np
import pytest

from paper_1411_3019_gb300 import inputs as I
from paper_1411_3019_gb300 import md

from parity_util import POS_100, assert_forces, oracle_run

pytestmark = pytest.mark.gpu


def _replicas(precision, nrep=6):
    return I.c4_replicas(nrep=nrep, seed=2, nmin=50, nmax=400, rmin=4.0, rmax=9.0, precision=precision, dt=0.002,
                         tol=1e-12 if precision == "fp64" else 1e-10)


def _run(systems, nsteps, engine, threads=None, per_launch=None, chunks=None):
    sim = md.Simulation(systems)
    sim.set_state(3)
    if engine:
        if threads:
            md.md_set_option(sim.h, md.MD_OPT_RESIDENT_THREADS, threads)
        if per_launch:
            md.md_set_option(sim.h, md.MD_OPT_RESIDENT_STEPS, per_launch)
        md.md_set_option(sim.h, md.MD_OPT_ENGINE, 1)
    for k in (chunks or [nsteps]):
        sim.step(k)
    sim.sync()
    st = sim.state()
    f, u = sim.forces()
    info = md.md_info(sim.h)
    sim.close()
    return st, f, u, info


def _same_bits(a, b):
    for key in ("x", "v", "p_half"):
        assert np.array_equal(a[0][key], b[0][key]), key
    assert np.array_equal(a[1], b[1])
    assert np.array_equal(a[2], b[2])


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_replicas_bit_identical_to_the_global_engine(precision):
    systems = _replicas(precision)
    g = _run(systems, 40, 0)
    r = _run(systems, 40, 1, per_launch=16)  # three launches: 16 + 16 + 8 steps
    _same_bits(g, r)
    assert r[3]["step"] == 43


def test_bonds_exclusions_and_partial_constraints_bit_identical():
    systems = I.c5_bead_molecules(nmol=80, beads=5, R=8.0, seed=4, precision="mixed", tol=1e-10)
    _same_bits(_run(systems, 30, 0), _run(systems, 30, 1))


def test_free_crowders_walls_and_periodic_box_bit_identical():
    systems = I.c3_bump_crowders(n_surf=600, n_free=1500, seed=5, precision="mixed", tol=1e-10)
    _same_bits(_run(systems, 25, 0), _run(systems, 25, 1, per_launch=10))


def test_linearly_smoothed_pairs_bit_identical():
    systems = _replicas("mixed", nrep=4)
    for sy in systems:
        sy["params"] = dict(sy["params"], pair_form=1, rcut=sy["params"]["rcut"] * 0 + 2.5)
    _same_bits(_run(systems, 20, 0), _run(systems, 20, 1))


@pytest.mark.parametrize("threads", [64, 128, 512])
def test_every_cta_size_gives_the_same_bits(threads):
    systems = _replicas("mixed", nrep=5)
    _same_bits(_run(systems, 20, 0), _run(systems, 20, 1, threads=threads))


def test_size_classes_of_a_wide_batch_give_the_same_bits():
    # sizes 96..1191: with 128-thread CTAs the registers allow six per SM and
    # shared memory three to eight, so the batch splits into several size
    # classes (one launch each per chunk); automatic CTA sizes as well
    systems = I.c4_replicas(nrep=24, seed=9, nmin=30, nmax=1500, rmin=4.0, rmax=16.0, precision="mixed",
                            dt=0.002, tol=1e-10)
    g = _run(systems, 12, 0)
    _same_bits(g, _run(systems, 12, 1, threads=128, per_launch=5))
    _same_bits(g, _run(systems, 12, 1, per_launch=5))


def test_resident_engine_matches_the_oracle():
    systems = _replicas("mixed", nrep=4)
    st, f, _, _ = _run(systems, 40, 1)
    ref = oracle_run(systems, 40, step0=3)[0]
    assert np.abs(st["x"] - ref["x"]).max() <= POS_100["mixed"]
    assert_forces(systems, st["x"], f, "mixed")


def test_switching_engines_mid_run_keeps_every_bit():
    systems = _replicas("mixed", nrep=4)
    ref = _run(systems, 30, 0)
    sim = md.Simulation(systems)
    sim.set_state(3)
    for engine, k in ((1, 10), (0, 7), (1, 13)):
        md.md_set_option(sim.h, md.MD_OPT_ENGINE, engine)
        sim.step(k)
    sim.sync()
    st = sim.state()
    f, u = sim.forces()
    res = sim.residual()
    sim.close()
    _same_bits(ref, (st, f, u))
    assert res["max_g_over_gradg"] < 1e-10


def test_profile_reports_the_resident_entries():
    sim = md.Simulation(_replicas("mixed", nrep=3))
    sim.set_state()
    md.md_set_option(sim.h, md.MD_OPT_ENGINE, 1)
    prof = md.md_profile_step(sim.h, 4)
    assert set(prof) == {"resident", "rebuild"} and prof["resident"] > 0
    assert md.md_info(sim.h)["step"] == 4
    sim.close()


def test_systems_the_resident_engine_cannot_hold_are_refused():
    big = [I.sphere_system(n=70000, R=120.0, seed=1, dmin=0.8, precision="mixed")]
    sim = md.Simulation(big)
    with pytest.raises(md.MdError, match="65535"):
        md.md_set_option(sim.h, md.MD_OPT_ENGINE, 1)
    assert md.md_get_option(sim.h, md.MD_OPT_ENGINE) == 0
    sim.close()
    free = [I.sphere_system(n=100, R=5.0, seed=2, precision="mixed", interacting=False)]
    sim = md.Simulation(free)
    with pytest.raises(md.MdError, match="pair interactions"):
        md.md_set_option(sim.h, md.MD_OPT_ENGINE, 1)
    sim.close()
    sim = md.Simulation(_replicas("mixed", nrep=2))
    for key, val in ((md.MD_OPT_ENGINE, 2), (md.MD_OPT_RESIDENT_THREADS, 100), (md.MD_OPT_RESIDENT_THREADS, 544),
                     (md.MD_OPT_RESIDENT_STEPS, 0)):
        with pytest.raises(md.MdError):
            md.md_set_option(sim.h, key, val)
    sim.close()
