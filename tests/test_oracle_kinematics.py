"""Pins of the oracle's kinematics with the thermostat off (gamma = 0):

* a free particle with no force moves on a straight line, x = x0 + v0 t,
  whatever its mass (Eq. 2: dx/dt = p/m);
* a particle held on a sphere with no force moves on a great circle at
  constant speed, x(t) = x0 cos(w t) + (v0/w) sin(w t), w = |v0| / R; the
  velocity Verlet + RATTLE trajectory approaches it as dt^2;
* setting a state projects the velocity on the tangent plane: n.v = 0 and
  v_in - v_out is parallel to n (Section 2.2: v.n = 0);
and of the noise-counter convention shared with the CUDA path: the random
force of the first step after a state set at step k0 is drawn at counter k0,
the next at k0 + 1 (a labelling choice, not a property of the method).
"""
import math

import numpy as np

from paper_1411_3019_gb300 import inputs as I


def test_free_particles_move_on_straight_lines(orc):
    m = 2.5
    prm = I.noninteracting(I.wca_params(dt=0.01, kT=0.0, gamma=0.0, mass=[m]))
    g = np.random.default_rng(1)
    x0 = g.uniform(-5, 5, (50, 3))
    v0 = g.standard_normal((50, 3))
    s = orc.System(None, prm, 50)
    s.set_state(x0, v0)
    s.step(300)
    st = s.state()
    np.testing.assert_allclose(st["x"], x0 + v0 * 3.0, rtol=0, atol=1e-12)
    np.testing.assert_allclose(st["v"], v0, rtol=0, atol=1e-14)


def _great_circle_error(orc, dt, T=2.0, R=3.0, m=1.7):
    prm = I.noninteracting(I.wca_params(dt=dt, kT=0.0, gamma=0.0, mass=[m], rattle_tol=1e-14))
    surf = {"kind": "sphere", "center": (0.0, 0.0, 0.0), "p": (R, 0, 0, 0)}
    g = np.random.default_rng(2)
    x0 = I.sample_surface(surf, 20, g)
    v = g.standard_normal((20, 3))
    v0 = v - (np.sum(v * x0, 1) / (R * R))[:, None] * x0
    s = orc.System(surf, prm, 20)
    s.set_state(x0, v0)
    nsteps = int(round(T / dt))
    s.step(nsteps)
    t = nsteps * dt
    w = np.linalg.norm(v0, axis=1) / R
    exact = x0 * np.cos(w * t)[:, None] + v0 / w[:, None] * np.sin(w * t)[:, None]
    st = s.state()
    speed_err = np.abs(np.linalg.norm(st["v"], axis=1) - np.linalg.norm(v0, axis=1)).max()
    return np.abs(st["x"] - exact).max(), speed_err


def test_free_motion_on_a_sphere_follows_great_circles(orc):
    e1, s1 = _great_circle_error(orc, 0.01)
    e2, s2 = _great_circle_error(orc, 0.005)
    assert e1 < 1e-3 and e2 < e1
    assert 3.0 < e1 / e2 < 5.0, (e1, e2)  # second order in dt
    assert s1 < 1e-3


def test_set_state_projects_velocities_on_the_tangent_plane(orc):
    surf = {"kind": "ellipsoid", "center": (1.0, 0.0, -1.0), "p": (6.0, 4.0, 3.0, 0.0)}
    prm = I.noninteracting(I.wca_params(dt=0.01))
    g = np.random.default_rng(3)
    x0 = I.sample_surface(surf, 30, g)
    v_in = g.standard_normal((30, 3)) * 2.0
    s = orc.System(surf, prm, 30)
    s.set_state(x0, v_in)
    v_out = s.state()["v"]
    for i in range(30):
        _, n = orc.surface_g(surf, prm, x0[i])
        assert abs(n @ v_out[i]) <= 1e-13 * np.linalg.norm(n) * max(1.0, np.linalg.norm(v_in[i]))
        assert np.linalg.norm(np.cross(v_in[i] - v_out[i], n)) <= 1e-12 * np.linalg.norm(n)
    assert s.residual()["max_n_dot_v"] < 1e-13


def test_noise_counter_convention(orc):
    m, kT, gamma, dt, k0 = 1.0, 1.0, 1.0, 0.01, 41
    prm = I.noninteracting(I.wca_params(dt=dt, kT=kT, gamma=gamma, seed=9, replica=2))
    x0 = np.zeros((1, 3))
    v0 = np.array([[0.3, -0.2, 0.1]])
    s = orc.System(None, prm, 1)
    s.set_state(x0, v0, step0=k0)
    s.step(1)
    amp = math.sqrt(2 * m * kT * gamma / dt)
    xi0 = orc.gauss3(9, 2, 0, k0) * amp
    xi1 = orc.gauss3(9, 2, 0, k0 + 1) * amp
    F0 = -gamma * m * v0[0] + xi0
    ph = m * v0[0] + 0.5 * dt * F0
    F1 = (-gamma * ph + 0.5 * (xi1 + xi0)) / (1 + 0.5 * gamma * dt)
    st = s.state()
    assert st["step"] == k0 + 1
    np.testing.assert_allclose(st["x"][0], dt / m * ph, rtol=1e-14, atol=1e-16)
    np.testing.assert_allclose(st["v"][0] * m, ph + 0.5 * dt * F1, rtol=1e-14, atol=1e-15)


def test_unconstrained_2d_plane_is_the_xy_projection_of_free_motion(orc):
    """The 2D baseline of the performance comparison (Section 3.1: particles in
    a plane with the z updates not evaluated): for non-interacting particles
    under Langevin noise, x and y follow exactly the x and y of free 3D
    motion with the same noise, z never moves and p_z stays 0."""
    g = np.random.default_rng(17)
    n = 40
    prm = I.noninteracting(I.wca_params(dt=0.002, gamma=1.0, kT=1.0, seed=9))
    x = np.column_stack([g.uniform(-5, 5, (n, 2)), np.full(n, 0.7)])
    v = g.normal(0, 1, (n, 3))
    flat = orc.System({"kind": "xy2d", "center": (0.0, 0.0, 0.7), "p": (0, 0, 0, 0)}, prm, n)
    flat.set_state(x, v)
    free = orc.System(None, prm, n)
    free.set_state(x, v)
    flat.step(40)
    free.step(40)
    a, b = flat.state(), free.state()
    assert np.array_equal(a["x"][:, :2], b["x"][:, :2])
    assert np.array_equal(a["p_half"][:, :2], b["p_half"][:, :2])
    assert np.all(a["x"][:, 2] == 0.7)
    assert np.all(a["v"][:, 2] == 0.0) and np.all(a["p_half"][:, 2] == 0.0)
    assert not np.all(b["x"][:, 2] == 0.7)
    assert flat.observables()["ndof"] == 2 * n
