"""Pins of the oracle's forces: the truncated-shifted LJ of Eq. (S1) at
points where its value is known, F = -dV/dx by central differences, Newton's
third law, zero force beyond the cutoff, the cell list against all pairs
(periodic images, exclusions, mixed cutoffs), and the bond and wall terms
(SI Section S3.2) by finite differences."""
import numpy as np
import pytest

from paper_1411_3019_gb300 import inputs as I

RNG = np.random.default_rng(7)


def _two(orc, r, prm=None):
    prm = prm or I.wca_params()
    x = np.array([[0.0, 0.0, 0.0], [r, 0.0, 0.0]])
    return orc.pair_forces(prm, x)


def test_wca_known_values(orc):
    f, u = _two(orc, 2 ** (1 / 6))
    assert np.abs(f).max() < 1e-12 and np.abs(u).max() < 1e-12
    f, u = _two(orc, 1.0)
    # phi(sigma) = 0, phi(r_c) = -eps: V(sigma) = eps; F(sigma) = 24 eps / sigma
    assert u.sum() == pytest.approx(1.0, rel=1e-14)
    assert f[0, 0] == pytest.approx(-24.0, rel=1e-14)
    assert f[1, 0] == pytest.approx(24.0, rel=1e-14)
    f, u = _two(orc, 1.2)
    assert np.abs(f).max() == 0.0 and np.abs(u).max() == 0.0


def test_lj_25_known_values(orc):
    prm = I.wca_params(ntypes=1)
    prm["eps"][0, 0] = 2.0
    prm["rcut"][0, 0] = 2.5
    r = 2 ** (1 / 6)
    f, u = _two(orc, r, prm)
    phic = 4 * 2.0 * (2.5 ** -12 - 2.5 ** -6)
    assert u.sum() == pytest.approx(-2.0 - phic, rel=1e-13)
    assert abs(f[0, 0]) < 1e-12


def _energy(orc, prm, x, types, mol):
    return orc.pair_forces(prm, x, types, mol)[1].sum()


@pytest.mark.parametrize("periodic", [(0, 0, 0), (1, 1, 0), (1, 1, 1)])
def test_forces_are_minus_energy_gradient(orc, periodic):
    prm = I.wca_params(ntypes=2, box_lo=(0, 0, 0), box_hi=(6.0, 6.5, 7.0), periodic=periodic)
    prm["eps"][1, 1] = 2.0
    prm["rcut"][1, 1] = 2.5
    prm["sigma"][0, 1] = prm["sigma"][1, 0] = 1.1
    prm["rcut"][0, 1] = prm["rcut"][1, 0] = 1.1 * 2 ** (1 / 6)
    n = 40
    g = np.random.default_rng(11)
    box = ((0.0, 0.0, 0.0), (6.0, 6.5, 7.0))
    x = I.rsa(lambda k, m: box[0] + g.random((m, 3)) * np.subtract(box[1], box[0]), [n], 0.9, g,
              periodic=periodic, box=box)[0]
    types = RNG.integers(0, 2, n).astype(np.int32)
    mol = np.arange(n, dtype=np.int32)
    f, _ = orc.pair_forces(prm, x, types, mol)
    for i in range(0, n, 5):
        for k in range(3):
            h = 1e-6
            xp, xm = x.copy(), x.copy()
            xp[i, k] += h
            xm[i, k] -= h
            d = -(_energy(orc, prm, xp, types, mol) - _energy(orc, prm, xm, types, mol)) / (2 * h)
            assert abs(d - f[i, k]) <= 1e-5 * max(1.0, abs(f[i, k])), (i, k, d, f[i, k])
    np.testing.assert_allclose(f.sum(0), 0.0, atol=1e-9 * max(1.0, np.abs(f).max()))


@pytest.mark.parametrize("case", ["open", "periodic", "excl"])
def test_cell_list_equals_all_pairs(orc, case):
    if case == "open":
        prm = I.wca_params(ntypes=2)
        prm["eps"][1, 1] = 2.0
        prm["rcut"][1, 1] = 2.5
        x = I.sample_surface({"kind": "sphere", "center": (0, 0, 0), "p": (12.0,)}, 1500,
                             np.random.default_rng(1))
        types = RNG.integers(0, 2, x.shape[0]).astype(np.int32)
        mol = np.arange(x.shape[0], dtype=np.int32)
    elif case == "periodic":
        prm = I.wca_params(box_lo=(-10, -10, -4), box_hi=(10, 10, 4), periodic=(1, 1, 0))
        x = RNG.uniform((-10, -10, -4), (10, 10, 4), (1500, 3))
        types = np.zeros(1500, np.int32)
        mol = np.arange(1500, dtype=np.int32)
    else:
        prm = I.wca_params(ntypes=5, exclude_intramol=1, beads_per_mol=5)
        prm["eps"][3, 3] = 2.0
        prm["rcut"][3, 3] = 2.5
        x = RNG.uniform(-6, 6, (1000, 3))
        types = np.tile(np.arange(5, dtype=np.int32), 200)
        mol = np.repeat(np.arange(200, dtype=np.int32), 5)
    fb, ub = orc.pair_forces(prm, x, types, mol, mode="brute")
    fc, uc = orc.pair_forces(prm, x, types, mol, mode="cells")
    scale = np.maximum(np.linalg.norm(fb, axis=1, keepdims=True), 1.0)
    assert np.max(np.abs(fb - fc) / scale) < 1e-12
    np.testing.assert_allclose(uc, ub, rtol=1e-12, atol=1e-12)
    assert np.abs(fb).max() > 0


def test_exclusions_remove_intramolecular_pairs(orc):
    prm = I.wca_params(exclude_intramol=1)
    x = np.array([[0.0, 0, 0], [1.0, 0, 0]])
    f, u = orc.pair_forces(prm, x, np.zeros(2, np.int32), np.array([4, 4], np.int32))
    assert np.abs(f).max() == 0 and np.abs(u).max() == 0
    f, u = orc.pair_forces(prm, x, np.zeros(2, np.int32), np.array([4, 5], np.int32))
    assert np.abs(f).max() > 0


def test_bond_and_wall_forces_match_energy_gradient(orc):
    prm = I.wca_params(beads_per_mol=5, bond_k=100.0, bond_r0=1.0, wall_enable=1,
                       wall_lo_z=-3.0, wall_hi_z=3.0, wall_eps=1.0, wall_sigma=1.0)
    n = 10
    x = np.zeros((n, 3))
    x[:, 0] = np.arange(n) * 1.05 + RNG.normal(0, 0.05, n)
    x[:, 1] = RNG.normal(0, 0.1, n)
    x[:, 2] = RNG.uniform(-2.4, 2.4, n)
    con = np.zeros(n, np.uint8)
    con[0] = 1
    f, u, bad = orc.bond_wall_forces(prm, x, con)
    assert bad == 0
    for i in range(n):
        for k in range(3):
            h = 1e-6
            xp, xm = x.copy(), x.copy()
            xp[i, k] += h
            xm[i, k] -= h
            d = -(orc.bond_wall_forces(prm, xp, con)[1].sum()
                  - orc.bond_wall_forces(prm, xm, con)[1].sum()) / (2 * h)
            assert abs(d - f[i, k]) <= 1e-5 * max(1.0, abs(f[i, k]))
    # bond energy without a factor 1/2, and no bond across molecules (4 -> 5)
    y = np.array([[0.0, 0, 0], [1.5, 0, 0]])
    _, u2, _ = orc.bond_wall_forces(dict(prm, wall_enable=0), y)
    assert u2.sum() == pytest.approx(100.0 * 0.25)
    y = np.zeros((6, 3))
    y[:, 0] = np.arange(6) * 2.0
    _, u6, _ = orc.bond_wall_forces(dict(prm, wall_enable=0), y)
    assert u6.sum() == pytest.approx(4 * 100.0 * 1.0)


def test_wall_known_value(orc):
    prm = I.wca_params(wall_enable=1, wall_lo_z=0.0, wall_hi_z=100.0, wall_eps=1.0, wall_sigma=1.0)
    x = np.array([[0.0, 0.0, 1.0]])
    f, u, _ = orc.bond_wall_forces(prm, x, np.zeros(1, np.uint8))
    assert u[0] == pytest.approx(4 * (1 - 1 + 0.25))
    assert f[0, 2] == pytest.approx(24.0)
    x = np.array([[0.0, 0.0, 2 ** (1 / 6)]])
    f, u, _ = orc.bond_wall_forces(prm, x, np.zeros(1, np.uint8))
    assert abs(u[0]) < 1e-12 and abs(f[0, 2]) < 1e-10


def test_periodic_forces_equal_explicit_image_sum(orc):
    """Periodic x, y: the minimum-image forces equal the forces of the
    central copy in an open system built from the 3x3 replicated box."""
    box = ((-4.5, -4.0, -3.0), (4.5, 4.0, 3.0))
    L = np.subtract(box[1], box[0])
    g = np.random.default_rng(21)
    n = 60
    x = I.rsa(lambda k, m: box[0] + g.random((m, 3)) * L, [n], 0.9, g,
              periodic=(1, 1, 0), box=box)[0]
    prm = I.wca_params(ntypes=1, box_lo=box[0], box_hi=box[1], periodic=(1, 1, 0))
    prm["eps"][0, 0] = 2.0
    prm["rcut"][0, 0] = 2.5
    f_per, u_per = orc.pair_forces(prm, x)
    reps = [x + np.array([i * L[0], j * L[1], 0.0]) for i in (-1, 0, 1) for j in (-1, 0, 1)]
    big = np.vstack(reps)
    open_prm = dict(prm, periodic=(0, 0, 0))
    f_big, u_big = orc.pair_forces(open_prm, big)
    centre = slice(4 * n, 5 * n)
    np.testing.assert_allclose(f_per, f_big[centre], rtol=1e-12, atol=1e-10)
    np.testing.assert_allclose(u_per, u_big[centre], rtol=1e-12, atol=1e-12)


def _lj25(form, eps=2.0):
    prm = I.wca_params(ntypes=1, pair_form=form)
    prm["eps"][0, 0] = eps
    prm["rcut"][0, 0] = 2.5
    return prm


def test_linearly_smoothed_lj_is_continuous_at_the_cutoff(orc):
    """The smoothed potential of the energy-conservation study: energy and force
    both vanish continuously at r_c (the energy quadratically in r_c - r), where
    the truncated-shifted force jumps by phi'(r_c) = -24 eps (2 (s/r_c)^12 -
    (s/r_c)^6) / r_c and its energy vanishes only linearly."""
    jump = abs(24 * 2.0 * (2 * 2.5 ** -12 - 2.5 ** -6) / 2.5)  # |phi'(r_c)| at eps = 2
    for delta in (1e-5, 1e-7):
        f_s, u_s = _two(orc, 2.5 - delta, _lj25(1))
        f_t, u_t = _two(orc, 2.5 - delta, _lj25(0))
        assert abs(u_t.sum()) == pytest.approx(jump * delta, rel=1e-3)
        assert abs(u_s.sum()) < 1e-3 * jump * delta
        assert abs(f_s[0, 0]) < 1e-3 * jump
        assert abs(f_t[0, 0]) == pytest.approx(jump, rel=1e-3)
    f, u = _two(orc, 2.5 + 1e-12, _lj25(1))
    assert np.abs(f).max() == 0.0 and np.abs(u).max() == 0.0


def test_smoothing_shifts_the_force_by_a_constant_and_vanishes_for_wca(orc):
    """V* - V = -(r - r_c) phi'(r_c): the force differs by the constant
    phi'(r_c) along the pair axis at every r; with the WCA cutoff phi'(r_c) = 0."""
    dphic = -24 * 2.0 * (2 * 2.5 ** -12 - 2.5 ** -6) / 2.5
    for r in (0.95, 1.1, 1.5, 2.0, 2.4):
        f_s, u_s = _two(orc, r, _lj25(1))
        f_t, u_t = _two(orc, r, _lj25(0))
        assert u_s.sum() - u_t.sum() == pytest.approx(-(r - 2.5) * dphic, rel=1e-12, abs=1e-15)
        # force on particle 1 (at +r along x) is +(-dV/dr)
        assert f_s[1, 0] - f_t[1, 0] == pytest.approx(dphic, rel=1e-12)
    for r in (0.9, 1.0, 1.1):
        f_s, u_s = _two(orc, r, I.wca_params(pair_form=1))
        f_t, u_t = _two(orc, r, I.wca_params(pair_form=0))
        np.testing.assert_allclose(f_s, f_t, rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(u_s, u_t, rtol=1e-12, atol=1e-12)


def test_smoothed_forces_are_minus_energy_gradient(orc):
    g = np.random.default_rng(21)
    prm = _lj25(1, eps=1.0)
    x = I.rsa(lambda k, m: g.uniform(-3.0, 3.0, (m, 3)), [60], 0.95, g)[0]
    f, _ = orc.pair_forces(prm, x)
    h = 1e-6
    for i in range(0, 60, 7):
        for k in range(3):
            xp, xm = x.copy(), x.copy()
            xp[i, k] += h
            xm[i, k] -= h
            fd = -(orc.pair_forces(prm, xp)[1].sum() - orc.pair_forces(prm, xm)[1].sum()) / (2 * h)
            assert f[i, k] == pytest.approx(fd, rel=1e-6, abs=1e-6)
