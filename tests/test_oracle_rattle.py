"""Pins of the oracle's RATTLE halves (Algorithm 1) against closed forms:
for the quadric surfaces g(y - a lambda n) = 0 is a quadratic in lambda whose
smaller root is the Newton answer; for the torus and the bump the root is
bracketed and bisected; the momentum half has the closed-form multiplier
mu = n.(p^{m+1/2} + dt/2 f) / (dt/2 n.n) (Section 2.2)."""
import math

import numpy as np
import pytest

from paper_1411_3019_gb300 import inputs as I

RNG = np.random.default_rng(2024)


def _prm(dt=0.002, tol=1e-12, **kw):
    p = I.wca_params(dt=dt, rattle_tol=tol, max_newton=30, **kw)
    return p


SURFS = {
    "sphere": {"kind": "sphere", "center": (1.0, -2.0, 0.5), "p": (10.0, 0, 0, 0)},
    "ellipsoid": {"kind": "ellipsoid", "center": (0.0, 1.0, 0.0), "p": (14.0, 9.0, 6.0, 0)},
    "plane": {"kind": "plane", "center": (0.0, 0.0, 3.0), "p": (0.3, -0.2, 1.0, 0)},
    "cylinder": {"kind": "cylinder", "center": (0.0, 0.0, 0.0), "p": (6.0, 2.0, 0, 0)},
    "torus": {"kind": "torus", "center": (0.0, 0.0, 0.0), "p": (10.0, 4.0, 0, 0)},
    "gaussian_bump": {"kind": "gaussian_bump", "center": (0.0, 0.0, 0.0), "p": (8.0, 5.0, 0, 0)},
}
BOX = ((-30.0, -30.0, -30.0), (30.0, 30.0, 30.0))


def _point_on(name):
    s = SURFS[name]
    if name == "plane":
        # a point of a tilted plane: choose x, y and solve the linear g for z
        a, b, c = s["p"][:3]
        x, y = RNG.uniform(-5, 5, 2)
        z = s["center"][2] - (a * x + b * y) / c
        return np.array([x, y, z])
    g = np.random.default_rng(RNG.integers(1 << 30))
    return I.sample_surface(s, 1, g, box=BOX)[0]


def _tangent_momentum(orc, name, prm, x, scale=1.0):
    _, n = orc.surface_g(SURFS[name], prm, x)
    v = RNG.standard_normal(3) * scale
    return v - (v @ n) / (n @ n) * n


def _prm_for(name, **kw):
    if name == "gaussian_bump":
        return _prm(box_lo=BOX[0], box_hi=BOX[1], periodic=(1, 1, 0), **kw)
    return _prm(**kw)


def _closed_form_lambda(name, x, y, a):
    s = SURFS[name]
    c = np.asarray(s["center"])
    if name == "sphere":
        n0 = 2 * (x - c)
        yy = y - c
        A, B, C = a * a * (n0 @ n0), -2 * a * (yy @ n0), yy @ yy - s["p"][0] ** 2
    elif name == "ellipsoid":
        ax = np.asarray(s["p"][:3])
        n0 = 2 * (x - c) / ax ** 2
        yy = y - c
        A = a * a * np.sum(n0 ** 2 / ax ** 2)
        B = -2 * a * np.sum(yy * n0 / ax ** 2)
        C = np.sum(yy ** 2 / ax ** 2) - 1
    elif name == "cylinder":
        ax = int(s["p"][1])
        m = np.ones(3)
        m[ax] = 0
        n0 = 2 * (x - c) * m
        yy = (y - c) * m
        A, B, C = a * a * (n0 @ n0), -2 * a * (yy @ n0), yy @ yy - s["p"][0] ** 2
    elif name == "plane":
        nrm = np.asarray(s["p"][:3])
        return (nrm @ (y - c)) / (a * (nrm @ nrm))
    # stable form: q = -(B + sign(B) sqrt(B^2 - 4AC)) / 2; roots q/A and C/q
    disc = math.sqrt(B * B - 4 * A * C)
    q = -0.5 * (B + math.copysign(disc, B))
    r1, r2 = q / A, C / q
    return r1 if abs(r1) < abs(r2) else r2


@pytest.mark.parametrize("name", ["sphere", "ellipsoid", "plane", "cylinder"])
@pytest.mark.parametrize("dt", [0.001, 0.01, 0.05])
def test_position_half_hits_quadric_root(orc, name, dt):
    prm = _prm_for(name, dt=dt)
    m = 1.7
    for _ in range(5):
        x = _point_on(name)
        p = _tangent_momentum(orc, name, prm, x, scale=2.0)
        f = RNG.standard_normal(3) * 20.0
        xn, ph, lam, its, st = orc.position_half(SURFS[name], prm, x, p, f, m)
        assert st in (0, 1), st
        a = dt * dt / (2 * m)
        y = x + dt / m * (p + 0.5 * dt * f)
        lam_ref = _closed_form_lambda(name, x, y, a)
        _, n0 = orc.surface_g(SURFS[name], prm, x)
        # the tolerance eta on positions fixes lambda to eta / (a |n0|)
        lam_tol = 10 * prm["rattle_tol"] / (a * np.linalg.norm(n0)) + 1e-12 * abs(lam_ref)
        assert abs(lam - lam_ref) <= lam_tol, (lam, lam_ref)
        g, n = orc.surface_g(SURFS[name], prm, xn)
        assert abs(g) / np.linalg.norm(n) < 1e-12
        # r_x = 0 at convergence: x^{m+1} = x^m + dt/m p^{m+1/2}
        np.testing.assert_allclose(xn, x + dt / m * ph, rtol=0, atol=1e-12)
        # p^{m+1/2} = p + dt/2 (f - lambda n(x^m))
        _, n0 = orc.surface_g(SURFS[name], prm, x)
        np.testing.assert_allclose(ph, p + 0.5 * dt * (f - lam * n0), rtol=0, atol=1e-12)
        assert its <= 6


@pytest.mark.parametrize("name", ["torus", "gaussian_bump"])
def test_position_half_hits_bisected_root(orc, name):
    prm = _prm_for(name, dt=0.01)
    m = 1.0
    for _ in range(6):
        x = _point_on(name)
        p = _tangent_momentum(orc, name, prm, x, scale=2.0)
        f = RNG.standard_normal(3) * 20.0
        xn, ph, lam, its, st = orc.position_half(SURFS[name], prm, x, p, f, m)
        assert st in (0, 1)
        a = prm["dt"] ** 2 / (2 * m)
        y = x + prm["dt"] / m * (p + 0.5 * prm["dt"] * f)
        _, n0 = orc.surface_g(SURFS[name], prm, x)

        def phi(lmb):
            return orc.surface_g(SURFS[name], prm, y - a * lmb * n0)[0]
        # bracket the root nearest 0 by stepping outwards from 0
        h = 1e-6 * (1 + abs(lam))
        lo, hi = -h, h
        for _ in range(200):
            if phi(lo) * phi(hi) <= 0:
                break
            lo, hi = lo * 2, hi * 2
        assert phi(lo) * phi(hi) <= 0
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            if phi(lo) * phi(mid) <= 0:
                hi = mid
            else:
                lo = mid
        lam_ref = 0.5 * (lo + hi)
        lam_tol = 10 * prm["rattle_tol"] / (a * np.linalg.norm(n0)) + 1e-12 * abs(lam_ref)
        assert abs(lam - lam_ref) <= lam_tol, (lam, lam_ref)


@pytest.mark.parametrize("name", list(SURFS))
def test_momentum_half_is_tangent_projection(orc, name):
    prm = _prm_for(name, dt=0.005)
    m = 2.5
    for _ in range(5):
        x = _point_on(name)
        ph = RNG.standard_normal(3) * 3.0
        f = RNG.standard_normal(3) * 30.0
        pn, mu, its, st = orc.momentum_half(SURFS[name], prm, x, ph, f, m)
        assert st in (0, 1)
        _, n = orc.surface_g(SURFS[name], prm, x)
        h = 0.5 * prm["dt"]
        q = ph + h * f
        mu_ref = (n @ q) / (h * (n @ n))
        assert abs(mu - mu_ref) <= 1e-10 * max(1.0, abs(mu_ref))
        np.testing.assert_allclose(pn, q - h * mu_ref * n, rtol=0, atol=1e-12)
        assert abs(n @ pn) / np.linalg.norm(n) <= 1e-13 * max(1.0, np.linalg.norm(pn))
        assert its <= 2


def test_position_half_reports_non_convergence(orc):
    name = "sphere"
    prm = _prm_for(name, dt=0.05)
    prm["max_newton"] = 1
    x = _point_on(name)
    p = _tangent_momentum(orc, name, prm, x, scale=5.0)
    f = RNG.standard_normal(3) * 50.0
    _, _, _, _, st = orc.position_half(SURFS[name], prm, x, p, f, 1.0)
    assert st == -1
    prm["max_newton"] = 30
    _, _, _, _, st = orc.position_half(SURFS[name], prm, x, p, f, 1.0)
    assert st in (0, 1)


def test_surface_gradients_match_finite_differences(orc):
    for name in SURFS:
        prm = _prm_for(name)
        for _ in range(4):
            x = _point_on(name) + RNG.standard_normal(3) * 0.3
            g0, n = orc.surface_g(SURFS[name], prm, x)
            for k in range(3):
                e = np.zeros(3)
                h = 1e-5 * max(1.0, abs(x[k]))
                e[k] = h
                gp = orc.surface_g(SURFS[name], prm, x + e)[0]
                gm = orc.surface_g(SURFS[name], prm, x - e)[0]
                assert abs((gp - gm) / (2 * h) - n[k]) <= 1e-6 * max(1.0, np.abs(n).max()), (name, k)


def test_surfaces_vanish_on_their_parametrisations(orc):
    """g = 0 on points drawn from each surface's parametric form (the
    samplers know nothing of g)."""
    for name in SURFS:
        prm = _prm_for(name)
        for _ in range(10):
            x = _point_on(name)
            g, n = orc.surface_g(SURFS[name], prm, x)
            assert abs(g) / np.linalg.norm(n) < 1e-12, name


def test_surface_signs(orc):
    prm = _prm()
    s = SURFS["sphere"]
    c = np.asarray(s["center"])
    g, _ = orc.surface_g(s, prm, c + np.array([0, 0, 11.0]))
    assert g == pytest.approx(121.0 - 100.0)
    g, _ = orc.surface_g(SURFS["torus"], prm, np.array([10.0, 0, 5.0]))
    assert g == pytest.approx(25.0 - 16.0)
    g, n = orc.surface_g(SURFS["ellipsoid"], prm, np.array([0.0, 1.0 + 9.0, 0.0]))
    assert g == pytest.approx(0.0, abs=1e-14)
    assert n[1] == pytest.approx(2.0 / 9.0)
