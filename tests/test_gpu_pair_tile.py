"""Cell-tiled pair kernel (MD_OPT_PAIR_TILE = 1: each warp takes a run of
sorted slots, split at cell boundaries; for each piece the home cell's
27-cell stencil is staged in shared memory and the piece's particles share
the lanes) against the oracle in both precisions, on workloads whose cells
hold one to several dozen particles: bead molecules on a spherical template
(bonds, exclusions, Lennard-Jones r_c = 2.5; runs spanning several cells), a
Gaussian bump with free crowders between walls (periodic x, y), and a dense
periodic Lennard-Jones lattice with r_c = 4 (64 particles per cell, shared
by several warps; stencils of 1,728 candidates, seven shared-memory windows),
at 8, 16 and 32 particles per warp.
Forces at the start and after a trajectory, the trajectory itself, and the
option's refusal where buckets are hashed."""
import numpy as np
import pytest

from paper_1411_3019_gb300 import inputs as I
from paper_1411_3019_gb300 import md

from parity_util import POS_100, assert_forces, gpu_run, oracle_run

pytestmark = pytest.mark.gpu

TILE = {md.MD_OPT_PAIR_TILE: 32}


def _tol(precision):
    return 1e-12 if precision == "fp64" else 1e-10


def _lattice(precision, k=12, rc=4.0, seed=3):
    """k^3 = 1,728 Lennard-Jones particles at density 0.79 in a periodic box
    of three cells of 4.33 along each axis at rc = 4: 64 particles per cell."""
    return I.lj_lattice(k, rc=rc, seed=seed, precision=precision, tol=_tol(precision))


def _check(systems, precision, nsteps, slots=32):
    opts = {md.MD_OPT_PAIR_TILE: slots}
    st0, f0, u0, _, _ = gpu_run(systems, 0, opts=opts)
    assert_forces(systems, st0["x"], f0, precision)
    _, _, u_ref, _, _ = oracle_run(systems, 0)
    np.testing.assert_allclose(u0.sum(), u_ref.sum(), rtol=1e-10 if precision == "fp64" else 1e-5)
    st, f, _, res, _ = gpu_run(systems, nsteps, opts=opts)
    ref = oracle_run(systems, nsteps)[0]
    assert np.abs(st["x"] - ref["x"]).max() <= POS_100[precision]
    assert_forces(systems, st["x"], f, precision)
    return st, res


@pytest.mark.parametrize("slots", [8, 16, 32])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_bead_molecules(precision, slots):
    systems = I.c5_bead_molecules(nmol=300, beads=5, R=10.0, seed=4, precision=precision, tol=_tol(precision))
    _check(systems, precision, 60, slots)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_bump_with_crowders_and_walls(precision):
    systems = I.c3_bump_crowders(n_surf=600, n_free=1500, seed=5, precision=precision, tol=_tol(precision))
    _, res = _check(systems, precision, 40)
    assert res["max_g_over_gradg"] < 10 * _tol(precision)


@pytest.mark.parametrize("slots", [8, 32])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_dense_lattice_with_several_windows(precision, slots):
    _check(_lattice(precision), precision, 30, slots)


def test_batch_of_systems_and_default_agree():
    """Several systems in one handle (cell ids offset per system): the tiled
    kernel's forces equal the default kernel's to float rounding."""
    reps = I.c4_replicas(nrep=3, seed=8, nmin=200, nmax=600, rmin=6.0, rmax=10.0, precision="fp64",
                         dt=0.002, tol=1e-12)
    for r in reps:  # systems of one batch share their pair table
        r["params"]["rcut"][0, 0] = 2.5
    systems = reps + _lattice("fp64", k=9, rc=2.5) + _lattice("fp64", k=10, rc=2.5, seed=4)
    a = gpu_run(systems, 20)
    b = gpu_run(systems, 20, opts=TILE)
    scale = np.maximum(np.linalg.norm(a[1], axis=1), 1.0)
    assert np.max(np.linalg.norm(a[1] - b[1], axis=1) / scale) < 1e-12
    assert np.abs(a[0]["x"] - b[0]["x"]).max() < 1e-10


def test_hashed_grid_refuses_the_tiled_kernel():
    """A sphere in a large open box: more than max(2^20, 4N) cells, so the
    buckets are hashed and the option is refused."""
    prm = I.wca_params(precision="mixed", box_lo=(-300.0,) * 3, box_hi=(300.0,) * 3)
    surf = {"kind": "sphere", "center": (0.0, 0.0, 0.0), "p": (8.0, 0.0, 0.0, 0.0)}
    g = I.rng(2, 9)
    x = I.rsa(lambda k, m: I.sample_surface(surf, m, g), [200], 1.0, g)[0]
    sim = md.Simulation([I._system("sphere_big_box", surf, prm, x, I.maxwell(200, 1.0, 1.0, g))])
    with pytest.raises(md.MdError):
        md.md_set_option(sim.h, md.MD_OPT_PAIR_TILE, 32)
    assert md.md_get_option(sim.h, md.MD_OPT_PAIR_TILE) == 0
    sim.close()
