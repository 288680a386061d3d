"""Pins of the oracle's time step (Algorithm S1) against what the paper and
the mathematics fix:

* the constraints g(x) = 0 and n.v = 0 hold after every step (Section 2.2);
* with gamma = 0 the scheme is velocity Verlet + RATTLE: the energy does not
  drift and its fluctuation scales as dt^2 (Section 3.1, energy test);
* the Langevin half-step momenta obey, for a free or plane-bound particle,
  q_{k+1} = a q_k + b (e_{k+1} + e_k) with a = (1-h)/(1+h), h = gamma dt/2,
  whose stationary variance is m kT/(1+h); the integer-step momenta have
  m kT (1 + h/2)/(1+h)^2. Both follow from the force combination of
  Algorithm S1 and pin its friction, its noise amplitude and its average;
* the mean squared displacement on a plane is the inertial Langevin form
  4D[t - tau(1 - e^{-t/tau})], which tends to 4Dt (SI Section S1.3) with
  D = kT tau / m;
* on a sphere <r0.rt>/R^2 = exp(-2 D t' / R^2) (SI Section S1.3), with the
  same inertial shift t' = t - tau(1 - e^{-t/tau});
* on a cylinder of radius R the MSD is 2Dt + 2R^2 (1 - e^{-Dt/R^2}) (SI
  Section S1.3); with inertia the arc-length displacement is Gaussian with
  variance s2(t) = 2D[t - tau(1 - e^{-t/tau})] (the tangential velocity is an
  Ornstein-Uhlenbeck process), so MSD = s2 + 2R^2 (1 - e^{-s2/(2R^2)}),
  which reduces to the SI's form for t >> tau;
* the temperature 2K/N_dof with 2 degrees of freedom per constrained
  particle equals the set kT (Section 3.1).
"""
import math

import numpy as np
import pytest

from paper_1411_3019_gb300 import inputs as I


def _free_system(orc, n, m, kT, gamma, dt, seed=5, surface=None, box=None):
    prm = I.noninteracting(I.wca_params(dt=dt, kT=kT, gamma=gamma, mass=[m], seed=seed,
                                        rattle_tol=1e-12))
    g = np.random.default_rng(seed)
    if surface is None:
        x = g.uniform(-50, 50, (n, 3))
    else:
        x = I.sample_surface(surface, n, g, box=box)
    v = g.standard_normal((n, 3)) * math.sqrt(kT / m)
    s = orc.System(surface, prm, n)
    s.set_state(x, v)
    return s, x


def test_constraints_hold_after_every_step(orc):
    sysd = I.sphere_system(n=300, R=6.0, seed=3, dmin=0.9, precision="fp64", dt=0.002, tol=1e-12)
    s = orc.System(sysd["surface"], sysd["params"], sysd["n"])
    s.set_state(sysd["x"], sysd["v"])
    for _ in range(40):
        assert s.step(1) == 0
        r = s.residual()
        assert r["max_g_over_gradg"] < 1e-12
        assert r["max_n_dot_v"] < 1e-12
    st = s.newton_stats()
    assert st["fail"] == 0
    assert st["iters"] <= 4 * 40 * 300


def _nve_energy_series(orc, dt, nsteps, every):
    sysd = I.sphere_system(n=150, R=6.0, seed=9, dmin=1.0, precision="fp64", dt=dt, tol=1e-13)
    prm = dict(sysd["params"], gamma=0.0, kT=0.0)
    s = orc.System(sysd["surface"], prm, sysd["n"])
    s.set_state(sysd["x"], sysd["v"])
    E = []
    for _ in range(nsteps // every):
        s.step(every)
        o = s.observables()
        E.append(o["kinetic"] + o["potential"])
    return np.array(E)


def test_nve_energy_is_conserved_with_dt2_fluctuations(orc):
    T = 6.0
    E1 = _nve_energy_series(orc, 0.004, int(T / 0.004), 25)
    E2 = _nve_energy_series(orc, 0.002, int(T / 0.002), 50)
    for E in (E1, E2):
        assert np.all(np.isfinite(E))
        assert np.std(E) / abs(np.mean(E)) < 2e-3
        # no secular drift: the two halves of the run agree within the noise
        h = len(E) // 2
        assert abs(E[h:].mean() - E[:h].mean()) < 3 * np.std(E) + 1e-12
    ratio = np.std(E1) / np.std(E2)
    assert 2.5 < ratio < 6.5, ratio


@pytest.mark.parametrize("where", ["free", "plane"])
def test_langevin_stationary_variances(orc, where):
    m, kT, gamma, dt = 2.0, 1.5, 1.0, 0.1
    h = gamma * dt / 2
    n = 3000
    if where == "free":
        s, _ = _free_system(orc, n, m, kT, gamma, dt)
        comps = [0, 1, 2]
    else:
        surf = {"kind": "plane", "center": (0.0, 0.0, 0.0), "p": (0.0, 0.0, 1.0, 0.0)}
        s, _ = _free_system(orc, n, m, kT, gamma, dt, surface=surf,
                            box=((-50, -50, 0), (50, 50, 0)))
        comps = [0, 1]
    s.step(100)
    ph, pi = [], []
    for _ in range(300):
        s.step(5)
        st = s.state()
        ph.append(st["p_half"][:, comps].ravel())
        pi.append((st["v"] * m)[:, comps].ravel())
    ph, pi = np.concatenate(ph), np.concatenate(pi)
    var_half = m * kT / (1 + h)
    var_int = m * kT * (1 + h / 2) / (1 + h) ** 2
    tol = 6 * var_half * math.sqrt(2.0 / (ph.size / 2))
    assert abs(ph.var() - var_half) < tol, (ph.var(), var_half)
    assert abs(pi.var() - var_int) < tol, (pi.var(), var_int)
    if where == "plane":
        st = s.state()
        assert np.abs(st["v"][:, 2]).max() < 1e-12
        assert np.abs(st["x"][:, 2]).max() < 1e-12


def test_plane_msd_follows_langevin_diffusion(orc):
    m, kT, gamma, dt = 1.0, 1.0, 1.0, 0.01
    D, tau = kT / (m * gamma), 1.0 / gamma
    surf = {"kind": "plane", "center": (0.0, 0.0, 0.0), "p": (0.0, 0.0, 1.0, 0.0)}
    n = 4000
    s, x0 = _free_system(orc, n, m, kT, gamma, dt, surface=surf, box=((-50, -50, 0), (50, 50, 0)))
    t = 0.0
    for t_check in (1.0, 4.0, 12.0):
        k = int(round((t_check - t) / dt))
        s.step(k)
        t += k * dt
        msd = s.observables()["msd"]
        theory = 4 * D * (t - tau * (1 - math.exp(-t / tau)))
        assert abs(msd / theory - 1) < 0.06, (t, msd, theory)
    # the late-time slope is 4D (the paper's plane law)
    s2_t, s2 = t, s.observables()["msd"]
    s.step(int(round(8.0 / dt)))
    slope = (s.observables()["msd"] - s2) / (8.0)
    assert abs(slope / (4 * D) - 1) < 0.2, slope


def test_sphere_correlation_decays_as_exp_minus_2Dt_over_R2(orc):
    m, kT, gamma, dt = 1.0, 1.0, 1.0, 0.02
    D, tau, R = kT / (m * gamma), 1.0 / gamma, 10.0
    surf = {"kind": "sphere", "center": (0.0, 0.0, 0.0), "p": (R, 0.0, 0.0, 0.0)}
    n = 3000
    s, _ = _free_system(orc, n, m, kT, gamma, dt, surface=surf)
    t = 0.0
    for t_check in (10.0, 25.0, 45.0):
        k = int(round((t_check - t) / dt))
        s.step(k)
        t += k * dt
        c = s.observables()["r0_dot_rt"]
        tp = t - tau * (1 - math.exp(-t / tau))
        theory = math.exp(-2 * D * tp / R ** 2)
        assert abs(c - theory) < 0.04, (t, c, theory)
        msd = s.observables()["msd"]
        assert abs(msd - 2 * R ** 2 * (1 - c)) < 1e-8 * R ** 2


def cylinder_msd(t, D, tau, R):
    s2 = 2 * D * (t - tau * (1 - math.exp(-t / tau)))
    return s2 + 2 * R ** 2 * (1 - math.exp(-s2 / (2 * R ** 2)))


def test_cylinder_msd_follows_the_closed_form(orc):
    m, kT, gamma, dt = 1.0, 1.0, 1.0, 0.01
    D, tau, R = kT / (m * gamma), 1.0 / gamma, 2.0
    surf = {"kind": "cylinder", "center": (0.0, 0.0, 0.0), "p": (R, 2.0, 0.0, 0.0)}
    n = 4000
    s, _ = _free_system(orc, n, m, kT, gamma, dt, surface=surf, box=((-3, -3, -50), (3, 3, 50)))
    t = 0.0
    for t_check in (1.0, 4.0, 10.0):
        k = int(round((t_check - t) / dt))
        s.step(k)
        t += k * dt
        msd = s.observables()["msd"]
        theory = cylinder_msd(t, D, tau, R)
        assert abs(msd / theory - 1) < 0.06, (t, msd, theory)
    # the circumferential part saturates at 2R^2: the late slope is that of the axis alone, 2D
    m2 = s.observables()["msd"]
    s.step(int(round(10.0 / dt)))
    slope = (s.observables()["msd"] - m2) / 10.0
    assert abs(slope / (2 * D) - 1) < 0.25, slope


def test_temperature_with_two_dof_per_constrained_particle(orc):
    sysd = I.sphere_system(n=400, R=9.0, seed=4, dmin=1.0, precision="fp64", dt=0.004, tol=1e-12)
    s = orc.System(sysd["surface"], sysd["params"], sysd["n"])
    s.set_state(sysd["x"], sysd["v"])
    s.step(500)
    kts = []
    for _ in range(60):
        s.step(20)
        o = s.observables()
        assert o["ndof"] == 2 * 400
        kts.append(o["kT"])
    h = 0.5 * sysd["params"]["gamma"] * sysd["params"]["dt"]
    expect = 1.0 * (1 + h / 2) / (1 + h) ** 2
    assert abs(np.mean(kts) - expect) < 0.03, (np.mean(kts), expect)


def test_force_modes_give_the_same_trajectory(orc):
    sysd = I.sphere_system(n=500, R=8.0, seed=8, dmin=0.9, precision="fp64", dt=0.002, tol=1e-12)
    out = []
    for mode in ("brute", "cells"):
        s = orc.System(sysd["surface"], sysd["params"], sysd["n"], force_mode=mode)
        s.set_state(sysd["x"], sysd["v"])
        s.step(20)
        out.append(s.state()["x"])
    np.testing.assert_allclose(out[0], out[1], rtol=0, atol=1e-11)


def test_first_force_after_set_state_reading(orc):
    """Reading: the first combined force is f - gamma p + f_r (no average)."""
    sysd = I.sphere_system(n=50, R=4.0, seed=2, dmin=1.0, precision="fp64")
    prm = sysd["params"]
    s = orc.System(sysd["surface"], prm, sysd["n"])
    s.set_state(sysd["x"], sysd["v"], step0=17)
    st = s.state()
    f, _ = s.forces()
    amp = math.sqrt(2 * 1.0 * prm["kT"] * prm["gamma"] / prm["dt"])
    fr = np.array([orc.gauss3(prm["seed"], prm["replica"], i, 17) for i in range(50)]) * amp
    np.testing.assert_allclose(st["F"], f - prm["gamma"] * st["v"] + fr, rtol=1e-13, atol=1e-12)
