"""Verlet neighbour list (md_set_neighbor_list) against the oracle, which
always searches a fresh cell list: trajectories and forces in both
precisions with a small skin (a rebuild every few steps) and a large one (a
rebuild every few tens), across md_step calls. Workloads: replicas on spheres,
bead molecules (bonds, exclusions, r_c = 2.5), a Gaussian bump with free
crowders between walls in a box periodic in x and y (particles cross the
boundary between builds). Also: a list too small for a particle's neighbours
is reported, a cell edge below r_c + skin is refused, the list can be
switched off mid-run, and a run repeats bit for bit."""
import numpy as np
import pytest

from paper_1411_3019_gb300 import inputs as I
from paper_1411_3019_gb300 import md

from parity_util import POS_100, assert_forces, oracle_run

pytestmark = pytest.mark.gpu


def _tol(precision):
    return 1e-12 if precision == "fp64" else 1e-10


def _cells(systems, skin):
    """Cell edge r_c + skin, as the list needs."""
    for s in systems:
        rc = float(np.max(s["params"]["rcut"]))
        s["params"] = dict(s["params"], cell_size=rc + skin)
    return systems


def _run(systems, skin, chunks, maxnb=64):
    sim = md.Simulation(systems)
    md.md_set_neighbor_list(sim.h, skin, maxnb)
    sim.set_state()
    for k in chunks:
        sim.step(k)
    sim.sync()
    st = sim.state()
    f, u = sim.forces()
    res = sim.residual()
    sim.close()
    return st, f, u, res


def _check(systems, precision, chunks, skin):
    st, f, _, res = _run(systems, skin, chunks)
    ref = oracle_run(systems, sum(chunks))[0]
    assert np.abs(st["x"] - ref["x"]).max() <= POS_100[precision]
    assert_forces(systems, st["x"], f, precision)
    return res


@pytest.mark.parametrize("skin", [0.05, 0.5])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_replicas_small_and_large_skin(precision, skin):
    systems = _cells(I.c4_replicas(nrep=3, seed=8, nmin=200, nmax=600, rmin=6.0, rmax=10.0, precision=precision,
                                   dt=0.002, tol=_tol(precision)), skin)
    res = _check(systems, precision, [37, 63], skin)
    assert res["max_g_over_gradg"] < 10 * _tol(precision)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_bead_molecules(precision):
    systems = _cells(I.c5_bead_molecules(nmol=300, beads=5, R=10.0, seed=4, precision=precision,
                                         tol=_tol(precision)), 0.4)
    _check(systems, precision, [60], 0.4)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_bump_with_crowders_periodic_and_walls(precision):
    systems = _cells(I.c3_bump_crowders(n_surf=600, n_free=1500, seed=5, precision=precision,
                                        tol=_tol(precision)), 0.3)
    _check(systems, precision, [20, 20], 0.3)


def test_list_too_small_is_reported():
    systems = _cells(I.lj_lattice(12, rc=2.5, seed=3, precision="mixed"), 0.3)
    sim = md.Simulation(systems)
    md.md_set_neighbor_list(sim.h, 0.3, 8)  # about 70 partners within 2.8 at density 0.79
    with pytest.raises(md.MdError) as e:
        sim.set_state()
        sim.step(1)
        sim.sync()
    assert e.value.code == md.MD_ERR_NLIST_FULL
    sim.close()


def test_cell_edge_below_cutoff_plus_skin_is_refused():
    systems = I.c4_replicas(nrep=2, seed=8, nmin=200, nmax=300, rmin=6.0, rmax=8.0, precision="mixed")
    sim = md.Simulation(systems)  # cell edge = the WCA cutoff
    with pytest.raises(md.MdError) as e:
        md.md_set_neighbor_list(sim.h, 0.3, 64)
    assert e.value.code == md.MD_ERR_INVALID_ARG
    sim.close()


def test_switch_off_mid_run_and_repeat_bit_for_bit():
    skin = 0.3
    systems = _cells(I.c4_replicas(nrep=2, seed=9, nmin=300, nmax=500, rmin=6.0, rmax=9.0, precision="mixed",
                                   dt=0.002, tol=1e-10), skin)
    a = _run(systems, skin, [25, 25])
    b = _run(systems, skin, [25, 25])
    for key in ("x", "v", "p_half"):
        assert np.array_equal(a[0][key], b[0][key]), key
    sim = md.Simulation(systems)
    md.md_set_neighbor_list(sim.h, skin, 64)
    sim.set_state()
    sim.step(25)
    md.md_set_neighbor_list(sim.h, 0.0, 64)
    sim.step(25)
    sim.sync()
    st = sim.state()
    sim.close()
    ref = oracle_run(systems, 50)[0]
    assert np.abs(st["x"] - ref["x"]).max() <= POS_100["mixed"]


def test_rebuild_counts():
    """The list is rebuilt only in steps where a particle has moved skin / 2:
    many rebuilds with a tiny skin, none in a few steps with a large one; a
    step is three launches (pair, integrate, the fused rebuild that returns
    at once without a rebuild), or seven with the separate rebuild kernels."""
    counts = {}
    for skin, steps in ((0.02, 40), (0.6, 5)):
        systems = _cells(I.c4_replicas(nrep=2, seed=9, nmin=300, nmax=500, rmin=6.0, rmax=9.0,
                                       precision="mixed", dt=0.002, tol=1e-10), skin)
        sim = md.Simulation(systems)
        md.md_set_neighbor_list(sim.h, skin, 64)
        sim.set_state()
        b0 = md.md_get_option(sim.h, md.MD_OPT_NLIST_BUILDS)
        sim.step(steps)
        fused = md.md_get_option(sim.h, md.MD_OPT_FUSED_REBUILD)
        assert fused == 1  # the cooperative launch is available on this GPU
        assert md.md_last_launch_count(sim.h) == 3 * steps
        counts[skin] = md.md_get_option(sim.h, md.MD_OPT_NLIST_BUILDS) - b0
        sim.close()
    assert counts[0.02] >= 5 and counts[0.6] == 0, counts


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_forces_after_set_state_and_resume_from_checkpoint(precision):
    """The headline workload's shape (ellipsoid + torus, 5,500 particles)
    with the list. Straight after md_set_state the list's forces equal those
    of a cell-list handle with the same cell edge to float rounding (same
    records; the list keeps the stencil's order of the pairs). A checkpoint
    restored with md_restore (which rebuilds the cell list and the list from
    the restored positions) repeats, bit for bit, a run that rebuilt its
    lists at the checkpoint step (switching the list on again rebuilds
    them). The forces straight after md_set_state and after the restored run
    match the oracle on every particle in both precisions."""
    skin = 0.3
    systems = _cells(I.c2_ellipsoid_torus(n_ell=4000, n_tor=1500, seed=8, precision=precision,
                                          tol=_tol(precision)), skin)
    with md.Simulation(systems) as cl:
        cl.set_state()
        f_cells, _ = cl.forces()
    with md.Simulation(systems) as a:
        md.md_set_neighbor_list(a.h, skin, 64)
        a.set_state()
        f0, _ = a.forces()
        assert_forces(systems, np.concatenate([sy["x"] for sy in systems]), f0, precision)
        sc = np.maximum(np.linalg.norm(f_cells, axis=1), 1.0)
        assert np.max(np.linalg.norm(f0 - f_cells, axis=1) / sc) < (1e-12 if precision == "fp64" else 1e-6)
        a.step(30)
        ck = a.state()
        md.md_set_neighbor_list(a.h, skin, 64)  # rebuild both lists at the checkpoint
        a.step(30)
        xa = a.state()
        fa, _ = a.forces()
    with md.Simulation(systems) as c:
        md.md_set_neighbor_list(c.h, skin, 64)
        c.set_state()
        md.md_restore(c.h, ck["x"], ck["p_half"], ck["step"])
        c.step(30)
        xc = c.state()
        fc, _ = c.forces()
    assert xc["step"] == 60
    for key in ("x", "p_half"):
        assert np.array_equal(xa[key], xc[key]), key
    assert np.array_equal(fa, fc)
    assert_forces(systems, xc["x"], fc, precision)


@pytest.mark.parametrize("workload", ["ellipsoid_torus", "bead_molecules"])
def test_queued_list_walk_gives_the_same_bits(workload):
    """The warp-queued list walk (default, at 32, 16 and 8 particles per
    warp) and the per-lane walk add each particle's terms in list order with
    the same arithmetic: forces and a trajectory across rebuilds agree bit for
    bit."""
    skin = 0.4
    if workload == "ellipsoid_torus":
        systems = _cells(I.c2_ellipsoid_torus(n_ell=4000, n_tor=1500, seed=8, precision="mixed"), skin)
    else:
        systems = _cells(I.c5_bead_molecules(nmol=400, beads=5, R=12.0, seed=6, precision="mixed"), skin)
    out = {}
    for queue, per_warp in ((1, 32), (0, 32), (1, 16), (1, 8)):
        with md.Simulation(systems) as sim:
            md.md_set_option(sim.h, md.MD_OPT_PAIR_QUEUE, queue)
            md.md_set_option(sim.h, md.MD_OPT_LIST_WARP, per_warp)
            assert md.md_get_option(sim.h, md.MD_OPT_PAIR_QUEUE) == queue
            assert md.md_get_option(sim.h, md.MD_OPT_LIST_WARP) == per_warp
            md.md_set_neighbor_list(sim.h, skin, 128)
            sim.set_state()
            f0, u0 = sim.forces()
            sim.step(40)
            sim.sync()
            out[(queue, per_warp)] = (f0, u0, sim.state(), md.md_get_option(sim.h, md.MD_OPT_NLIST_BUILDS))
    ref = out[(0, 32)]
    assert ref[3] > 1  # rebuilds inside the run
    for key_run, run in out.items():
        assert np.array_equal(run[0], ref[0]) and np.array_equal(run[1], ref[1]), key_run
        for key in ("x", "p_half"):
            assert np.array_equal(run[2][key], ref[2][key]), (key_run, key)


@pytest.mark.parametrize("workload", ["ellipsoid_torus", "bead_molecules"])
def test_fused_rebuild_gives_the_same_bits(workload):
    """The fused rebuild (one cooperative launch with grid barriers) and the
    five separate rebuild kernels build the same cell list and Verlet list:
    trajectories across many rebuilds agree bit for bit, and so do the build
    counts; the separate form launches seven kernels per step."""
    skin = 0.1
    if workload == "ellipsoid_torus":
        systems = _cells(I.c2_ellipsoid_torus(n_ell=4000, n_tor=1500, seed=8, precision="mixed"), skin)
    else:
        systems = _cells(I.c5_bead_molecules(nmol=400, beads=5, R=12.0, seed=6, precision="mixed"), skin)
    out = {}
    for fused in (1, 0):
        with md.Simulation(systems) as sim:
            md.md_set_option(sim.h, md.MD_OPT_FUSED_REBUILD, fused)
            md.md_set_neighbor_list(sim.h, skin, 128)
            sim.set_state()
            b0 = md.md_get_option(sim.h, md.MD_OPT_NLIST_BUILDS)
            sim.step(60)
            launches = md.md_last_launch_count(sim.h)
            sim.sync()
            out[fused] = (sim.state(), sim.forces()[0], md.md_get_option(sim.h, md.MD_OPT_NLIST_BUILDS) - b0)
            assert md.md_get_option(sim.h, md.MD_OPT_FUSED_REBUILD) == fused
            assert launches == (3 if fused else 7) * 60
    assert out[1][2] == out[0][2] > 5
    assert np.array_equal(out[1][1], out[0][1])
    for key in ("x", "p_half"):
        assert np.array_equal(out[1][0][key], out[0][0][key]), key


@pytest.mark.parametrize("fused", [1, 0])
def test_stored_noise_gives_the_same_bits(fused):
    """The integrator's stored unit normals (MD_OPT_STORE_NOISE = 1, read back
    by the next step's force combination) against drawing both steps' normals
    every step: the same trajectory bit for bit, through a restore from a
    checkpoint (after which the first step draws both again), with the fused
    rebuild and with the separate rebuild kernels (each advances the step
    counter and records the stored step)."""
    skin = 0.2
    systems = _cells(I.c2_ellipsoid_torus(n_ell=4000, n_tor=1500, seed=9, precision="mixed"), skin)
    out = {}
    for store in (1, 0):
        with md.Simulation(systems) as sim:
            md.md_set_option(sim.h, md.MD_OPT_FUSED_REBUILD, fused)
            md.md_set_option(sim.h, md.MD_OPT_STORE_NOISE, store)
            assert md.md_get_option(sim.h, md.MD_OPT_STORE_NOISE) == store
            md.md_set_neighbor_list(sim.h, skin, 128)
            sim.set_state()
            sim.step(25)
            sim.sync()
            chk = sim.state()
            sim.step(15)
            sim.sync()
            md.md_restore(sim.h, chk["x"], chk["p_half"], chk["step"])
            sim.step(30)
            sim.sync()
            out[store] = sim.state()
    for key in ("x", "p_half"):
        assert np.array_equal(out[1][key], out[0][key]), key
    assert out[1]["step"] == 55
