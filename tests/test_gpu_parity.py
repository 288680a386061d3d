"""GPU (CUDA, through the C ABI) against the oracle on the same seeded
inputs: forces, one step, 100 steps, every surface kind, batches of
replicas, bonds/exclusions/partial constraints, walls with periodic x, y,
constraint residuals and observables."""
import numpy as np
import pytest

from paper_1411_3019_gb300 import inputs as I

from parity_util import POS_100, assert_forces, gpu_run, oracle_run

pytestmark = pytest.mark.gpu


def _c1(precision, n=1000):
    tol = 1e-12 if precision == "fp64" else 1e-10
    return [I.sphere_system(n=n, R=10.0, seed=1, dmin=0.8, precision=precision, dt=0.001, tol=tol)]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_forces_match_oracle_on_the_plain_workload(precision):
    systems = _c1(precision)
    st, f, u, res, _ = gpu_run(systems, 0)
    _, f_ref, u_ref, _, _ = oracle_run(systems, 0)
    assert_forces(systems, st["x"], f, precision)
    np.testing.assert_allclose(u.sum(), u_ref.sum(), rtol=1e-10 if precision == "fp64" else 1e-5)
    assert np.abs(f_ref).max() > 10.0  # overlapping start: a real test of the pair kernel


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("nsteps", [1, 2, 100])
def test_trajectory_matches_oracle(precision, nsteps):
    systems = _c1(precision)
    st, f, u, res, obs = gpu_run(systems, nsteps, step0=7)
    ref, f_ref, _, res_ref, obs_ref = oracle_run(systems, nsteps, step0=7)
    dx = np.abs(st["x"] - ref["x"]).max()
    dv = np.abs(st["v"] - ref["v"]).max()
    assert dx <= POS_100[precision], dx
    assert dv <= 1e3 * POS_100[precision], dv
    if nsteps > 1:
        assert np.abs(st["p_half"] - ref["p_half"]).max() <= 1e3 * POS_100[precision]
    assert st["step"] == 7 + nsteps
    tol = systems[0]["params"]["rattle_tol"]
    assert res["max_g_over_gradg"] < tol
    # both precisions project p^k with the float64 normal
    assert res["max_n_dot_v"] < 1e-9
    assert_forces(systems, st["x"], f, precision)
    assert obs[0]["ndof"] == 2 * systems[0]["n"]
    assert obs[0]["kT"] == pytest.approx(obs_ref[0]["kT"], rel=1e-6)


SURFACES = {
    "plane": ({"kind": "plane", "center": (0.0, 0.0, 0.0), "p": (0.0, 0.0, 1.0, 0.0)},
              dict(box_lo=(-12, -12, -3), box_hi=(12, 12, 3), periodic=(1, 1, 0))),
    "sphere": ({"kind": "sphere", "center": (1.0, 2.0, -1.0), "p": (8.0, 0, 0, 0)}, {}),
    "ellipsoid": ({"kind": "ellipsoid", "center": (0.0, 0.0, 0.0), "p": (11.0, 8.0, 6.0, 0)}, {}),
    "torus": ({"kind": "torus", "center": (0.0, 0.0, 0.0), "p": (10.0, 4.0, 0, 0)}, {}),
    "gaussian_bump": ({"kind": "gaussian_bump", "center": (0.0, 0.0, 0.0), "p": (6.0, 5.0, 0, 0)},
                      dict(box_lo=(-15, -15, -4), box_hi=(15, 15, 10), periodic=(1, 1, 0))),
    "cylinder": ({"kind": "cylinder", "center": (0.0, 0.0, 0.0), "p": (5.0, 2.0, 0, 0)},
                 dict(box_lo=(-8, -8, -10), box_hi=(8, 8, 10), periodic=(0, 0, 1))),
}


def _surface_system(name, precision, n=300, seed=3):
    surf, extra = SURFACES[name]
    prm = I.wca_params(precision=precision, dt=0.002, rattle_tol=1e-12 if precision == "fp64" else 1e-10,
                       seed=seed, **extra)
    g = I.rng(seed, 11)
    box = (prm["box_lo"], prm["box_hi"]) if extra else None
    x = I.rsa(lambda k, m: I.sample_surface(surf, m, g, box=box), [n], 0.95, g,
              periodic=prm["periodic"], box=box)[0]
    return [I._system(name, surf, prm, x, I.maxwell(n, 1.0, 1.0, g))]


@pytest.mark.parametrize("name", list(SURFACES))
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_every_surface_matches_oracle(name, precision):
    systems = _surface_system(name, precision)
    st, f, u, res, _ = gpu_run(systems, 50)
    ref, f_ref, _, res_ref, _ = oracle_run(systems, 50)
    assert np.abs(st["x"] - ref["x"]).max() <= POS_100[precision]
    assert_forces(systems, st["x"], f, precision)
    assert res["max_g_over_gradg"] < systems[0]["params"]["rattle_tol"]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batch_of_replicas_matches_independent_oracles(precision):
    systems = I.c4_replicas(nrep=6, seed=2, nmin=50, nmax=400, rmin=4.0, rmax=9.0, precision=precision,
                            dt=0.002, tol=1e-12 if precision == "fp64" else 1e-10)
    st, f, u, res, obs = gpu_run(systems, 40)
    ref, f_ref, _, _, obs_ref = oracle_run(systems, 40)
    assert np.abs(st["x"] - ref["x"]).max() <= POS_100[precision]
    assert_forces(systems, st["x"], f, precision)
    assert len(obs) == 6
    for a, b, sy in zip(obs, obs_ref, systems):
        assert a["n"] == sy["n"]
        assert a["msd"] == pytest.approx(b["msd"], rel=1e-5, abs=1e-9)
        assert a["r0_dot_rt"] == pytest.approx(b["r0_dot_rt"], rel=1e-6)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_bead_molecules_match_oracle(precision):
    systems = I.c5_bead_molecules(nmol=300, beads=5, R=10.0, seed=4, precision=precision,
                                  tol=1e-12 if precision == "fp64" else 1e-10)
    st, f, u, res, obs = gpu_run(systems, 60)
    ref, f_ref, u_ref, _, obs_ref = oracle_run(systems, 60)
    assert np.abs(st["x"] - ref["x"]).max() <= POS_100[precision]
    assert_forces(systems, st["x"], f, precision)
    np.testing.assert_allclose(u.sum(), u_ref.sum(), rtol=1e-9 if precision == "fp64" else 1e-5)
    con = systems[0]["constrained"].astype(bool)
    assert obs[0]["ndof"] == 2 * con.sum() + 3 * (~con).sum()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_constrained_and_free_with_walls_match_oracle(precision):
    systems = I.c3_bump_crowders(n_surf=600, n_free=1500, seed=5, precision=precision,
                                 tol=1e-12 if precision == "fp64" else 1e-10)
    st, f, u, res, _ = gpu_run(systems, 40)
    ref, f_ref, _, _, _ = oracle_run(systems, 40)
    assert np.abs(st["x"] - ref["x"]).max() <= POS_100[precision]
    assert_forces(systems, st["x"], f, precision)


def test_mixed_tracks_fp64_within_tolerance():
    a = gpu_run(_c1("fp64"), 100)[0]
    b = gpu_run(_c1("mixed"), 100)[0]
    assert np.abs(a["x"] - b["x"]).max() <= POS_100["mixed"]


@pytest.mark.parametrize("frozen", [0, 1])
def test_frozen_normal_reaches_the_same_root(frozen):
    systems = _surface_system("torus", "fp64")
    systems[0]["params"] = dict(systems[0]["params"], frozen_normal=frozen)
    st = gpu_run(systems, 30)[0]
    ref = oracle_run(systems, 30)[0]
    assert np.abs(st["x"] - ref["x"]).max() <= POS_100["fp64"]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("form", [0, 1])
def test_lj_cutoff_25_in_both_pair_forms_matches_oracle(precision, form):
    """Truncated-shifted (Eq. S1) and linearly smoothed LJ at r_c = 2.5 sigma,
    where the two forms differ: forces at the start and after 50 steps."""
    prm = I.wca_params(precision=precision, dt=0.002, rattle_tol=1e-12 if precision == "fp64" else 1e-10,
                       seed=6, pair_form=form)
    prm["rcut"][0, 0] = 2.5
    surf = {"kind": "sphere", "center": (0.0, 0.0, 0.0), "p": (9.0, 0, 0, 0)}
    g = I.rng(6, 11)
    x = I.rsa(lambda k, m: I.sample_surface(surf, m, g), [500], 0.95, g)[0]
    systems = [I._system("lj25", surf, prm, x, I.maxwell(500, 1.0, 1.0, g))]
    st0, f0, u0, _, _ = gpu_run(systems, 0)
    assert_forces(systems, st0["x"], f0, precision)
    _, _, u_ref, _, _ = oracle_run(systems, 0)
    np.testing.assert_allclose(u0.sum(), u_ref.sum(), rtol=1e-10 if precision == "fp64" else 1e-5)
    st, f, u, res, _ = gpu_run(systems, 50)
    ref = oracle_run(systems, 50)[0]
    assert np.abs(st["x"] - ref["x"]).max() <= POS_100[precision]
    assert_forces(systems, st["x"], f, precision)
