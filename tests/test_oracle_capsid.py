"""Pins of the oracle's capsid-model terms (SI Section S3.2): the bend angle
V = k_a (theta - theta0)^2 at a right angle and on a straight chain (closed
forms), bond rest lengths from the bead types, the spherical Lennard-Jones
wall at a point where its value is known, Newton's third law, and every
force against central differences of the energy."""
import math

import numpy as np
import pytest

from paper_1411_3019_gb300 import inputs as I

KA = 250.0


def _chain_params(**over):
    prm = I.wca_params(ntypes=4)
    prm["rcut"][:, :] = 0.0  # bonded terms only
    prm.update(beads_per_mol=3, bond_k=0.0, bond_r0=1.0, angle_k=KA, angle_theta0=math.pi)
    prm.update(over)
    return prm


def test_right_angle_energy_and_forces(orc):
    x = np.array([[1.0, 0.0, 0.0], [0.0, 0.0, 0.0], [0.0, 1.0, 0.0]])
    f, u, bad = orc.bond_wall_forces(_chain_params(), x)
    assert not bad
    # theta = pi/2: V = k (pi/2)^2, split in thirds
    np.testing.assert_allclose(u, [KA * math.pi ** 2 / 12] * 3, rtol=1e-14)
    # dV/dtheta = -k pi; the end beads are pushed perpendicular to their bond,
    # away from each other (opening the angle); the middle bead takes the rest
    np.testing.assert_allclose(f[0], [0.0, -KA * math.pi, 0.0], atol=1e-12)
    np.testing.assert_allclose(f[2], [-KA * math.pi, 0.0, 0.0], atol=1e-12)
    np.testing.assert_allclose(f[1], [KA * math.pi, KA * math.pi, 0.0], atol=1e-12)


def test_straight_chain_is_at_rest_and_bent_chain_is_not(orc):
    x = np.array([[-1.3, 0.0, 0.0], [0.0, 0.0, 0.0], [0.9, 0.0, 0.0]])
    f, u, _ = orc.bond_wall_forces(_chain_params(), x)
    assert np.abs(f).max() < 1e-12 and np.abs(u).max() < 1e-20
    x[2, 1] = 1e-3  # slightly bent: restoring force towards the line
    f, u, _ = orc.bond_wall_forces(_chain_params(), x)
    assert f[2, 1] < 0 and u.sum() > 0


def test_third_law_and_energy_split(orc):
    g = np.random.default_rng(3)
    x = np.cumsum(g.normal(0, 0.6, (12, 3)) + [1.0, 0.0, 0.0], axis=0)
    prm = _chain_params(beads_per_mol=4, bond_k=50.0, bond_r0=1.0, angle_theta0=2.5)
    f, u, _ = orc.bond_wall_forces(prm, x)
    np.testing.assert_allclose(f.sum(axis=0), 0.0, atol=1e-9)
    # one molecule alone carries the same energy as in the batch of three
    for m in range(3):
        _, um, _ = orc.bond_wall_forces(prm, x[4 * m:4 * m + 4])
        assert um.sum() == pytest.approx(u[4 * m:4 * m + 4].sum(), rel=1e-13)


def test_bond_rest_length_from_the_bead_types(orc):
    sig = np.array([1.0, 1.35, 1.75, 1.0])
    prm = _chain_params(beads_per_mol=2, angle_k=0.0, bond_k=50.0, bond_r0_mix=1)
    prm["sigma"] = 0.5 * (sig[:, None] + sig[None, :])
    types = np.array([1, 2], np.int32)
    r0 = 2 ** (1 / 6) * (1.35 + 1.75) / 4  # the SI's r_0,ij
    for dr, expect in ((0.0, 0.0), (0.01, 2 * 50.0 * 0.01), (-0.02, -2 * 50.0 * 0.02)):
        x = np.array([[0.0, 0.0, 0.0], [r0 + dr, 0.0, 0.0]])
        f, u, _ = orc.bond_wall_forces(prm, x, type_=types)
        # force on bead 1 is -dV/dr = -2k (r - r0)
        assert f[1, 0] == pytest.approx(-expect, abs=1e-12)
        assert u.sum() == pytest.approx(50.0 * dr * dr, abs=1e-15)


def test_spherical_wall_known_values(orc):
    prm = _chain_params(beads_per_mol=0, angle_k=0.0, wall_enable=1, wall_kind=1, wall_radius=5.0,
                        wall_center=(1.0, -2.0, 0.5), wall_eps=1.0, wall_sigma=1.0)
    c = np.array([1.0, -2.0, 0.5])
    d = np.array([2.0, -1.0, 2.0]) / 3.0  # unit vector
    # at r - R_w = sigma_w: V = eps (4 (1 - 1) + 1), force 24 eps / sigma_w outward
    f, u, bad = orc.bond_wall_forces(prm, (c + 6.0 * d)[None, :], np.zeros(1, np.uint8))
    assert not bad
    assert u[0] == pytest.approx(1.0, rel=1e-14)
    np.testing.assert_allclose(f[0], 24.0 * d, rtol=1e-13)
    # beyond 2^(1/6) sigma_w: nothing; constrained particles: nothing; behind: flagged
    f, u, _ = orc.bond_wall_forces(prm, (c + (5.0 + 1.13) * d)[None, :], np.zeros(1, np.uint8))
    assert np.abs(f).max() == 0.0 and u[0] == 0.0
    f, u, _ = orc.bond_wall_forces(prm, (c + 6.0 * d)[None, :], np.ones(1, np.uint8))
    assert np.abs(f).max() == 0.0
    _, _, bad = orc.bond_wall_forces(prm, (c + 4.0 * d)[None, :], np.zeros(1, np.uint8))
    assert bad


def test_capsid_terms_are_minus_energy_gradient(orc):
    g = np.random.default_rng(5)
    sig = np.array([1.0, 1.35, 1.75, 1.0])
    prm = _chain_params(beads_per_mol=4, bond_k=50.0, bond_r0_mix=1, angle_theta0=math.pi,
                        wall_enable=1, wall_kind=1, wall_radius=2.0, wall_center=(0.0, 0.0, 0.0),
                        wall_eps=1.0, wall_sigma=1.0)
    prm["sigma"] = 0.5 * (sig[:, None] + sig[None, :])
    nmol = 3
    base = g.normal(0, 1, (nmol, 3))
    base = 3.5 * base / np.linalg.norm(base, axis=1, keepdims=True)
    x = np.concatenate([b + np.cumsum(g.normal(0, 0.3, (4, 3)) + 0.9 * b / 3.5, axis=0) for b in base])
    types = np.tile(np.arange(4, dtype=np.int32), nmol)
    con = np.tile(np.array([1, 0, 0, 0], np.uint8), nmol)
    f, u, bad = orc.bond_wall_forces(prm, x, con, type_=types)
    assert not bad
    h = 1e-6
    for i in range(x.shape[0]):
        for k in range(3):
            xp, xm = x.copy(), x.copy()
            xp[i, k] += h
            xm[i, k] -= h
            fd = -(orc.bond_wall_forces(prm, xp, con, type_=types)[1].sum()
                   - orc.bond_wall_forces(prm, xm, con, type_=types)[1].sum()) / (2 * h)
            assert f[i, k] == pytest.approx(fd, rel=1e-6, abs=1e-5)


def test_spherical_wall_is_minus_energy_gradient(orc):
    g = np.random.default_rng(8)
    prm = _chain_params(beads_per_mol=0, angle_k=0.0, wall_enable=1, wall_kind=1, wall_radius=4.0,
                        wall_center=(0.5, 0.0, -1.0), wall_eps=2.0, wall_sigma=1.2)
    d = g.normal(0, 1, (6, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    x = np.array([0.5, 0.0, -1.0]) + (4.0 + g.uniform(0.9, 1.3, (6, 1))) * d
    con = np.zeros(6, np.uint8)
    f, u, bad = orc.bond_wall_forces(prm, x, con)
    assert not bad and u.sum() > 0
    h = 1e-6
    for i in range(6):
        for k in range(3):
            xp, xm = x.copy(), x.copy()
            xp[i, k] += h
            xm[i, k] -= h
            fd = -(orc.bond_wall_forces(prm, xp, con)[1].sum() - orc.bond_wall_forces(prm, xm, con)[1].sum()) / (2 * h)
            assert f[i, k] == pytest.approx(fd, rel=1e-6, abs=1e-6)
