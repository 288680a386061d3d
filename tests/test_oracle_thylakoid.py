"""Pins of the oracle's thylakoid composite (SI S3.1; the assembly of the
pieces is a reading stated in the oracle): points placed on every piece by
its own parametrisation satisfy g = 0 under the oracle's piece selection;
the tangent planes of adjacent pieces agree across every kind of junction
(face plane and connector rim, connector and bridge, plane and corner
cylinder); particles diffusing over the surface cross the junctions and stay
on it (position half of Algorithm 1 on the piece selected at x^m)."""
import math

import numpy as np
import pytest

from paper_1411_3019_gb300 import inputs as I

RB, LX, RC, LB, LZ = 1.5, 15.0, 3.0, 10.0, 30.0


def _prm(**over):
    return I.wca_params(box_lo=(-45.0, -14.0, -LZ / 2), box_hi=(45.0, 14.0, LZ / 2), periodic=(0, 0, 1),
                        rattle_tol=1e-12, **over)


def _g(orc, surf, x):
    g, n = orc.surface_g(surf, _prm(), np.asarray(x, float))
    return g, n


def test_points_on_every_piece_satisfy_g(orc):
    surf = I.thylakoid_surface(RB, LX, RC, LB, center=(0.5, -1.0, 2.0))
    x = I.sample_thylakoid(surf, 6000, np.random.default_rng(2), LZ)
    worst = max(abs(g) / np.linalg.norm(n) for g, n in (_g(orc, surf, xi) for xi in x))
    assert worst < 1e-12
    # every piece is represented: bridge, connectors, face and side planes, corners
    xc = surf["center"][0]
    assert np.any(np.abs(x[:, 0] - xc) < LB / 2 - 0.1)
    assert np.any((np.abs(x[:, 0] - xc) > LB / 2 + 0.1) & (np.abs(x[:, 0] - xc) < LB / 2 + RC - 0.1))


def _parallel(n1, n2):
    return np.linalg.norm(np.cross(n1, n2)) / (np.linalg.norm(n1) * np.linalg.norm(n2))


@pytest.mark.parametrize("phi", [0.3, 1.9, 4.0])
def test_tangent_planes_agree_across_the_junctions(orc, phi):
    surf = I.thylakoid_surface(RB, LX, RC, LB)
    x0L = -LB / 2
    xfL = x0L - RC
    e = 1e-7
    c, s = math.cos(phi), math.sin(phi)
    rout = RB + RC
    pairs = [
        # face plane | connector rim (r = R_b + R_c at x = x_face)
        ([xfL - e, rout * c, rout * s], [xfL + e, (rout - e) * c, (rout - e) * s]),
        # connector | bridge (r = R_b at the bridge end)
        ([x0L - e, RB * c, RB * s], [x0L + e, RB * c, RB * s]),
        # face plane | corner cylinder of the left block
        ([xfL, LX / 2 - e, 3.0 * s], [xfL - e, LX / 2 + e, 3.0 * s]),
        # corner cylinder | top plane of the left block
        ([xfL - RC + e, LX / 2 + RC, 1.0], [xfL - RC - e, LX / 2 + RC, 1.0]),
    ]
    for a, b in pairs:
        ga, na = _g(orc, surf, a)
        gb, nb = _g(orc, surf, b)
        assert abs(ga) / np.linalg.norm(na) < 1e-6 and abs(gb) / np.linalg.norm(nb) < 1e-6, (a, b, ga, gb)
        assert _parallel(na, nb) < 1e-5, (a, b, na, nb)


def test_diffusion_crosses_junctions_and_stays_on_the_surface(orc):
    surf = I.thylakoid_surface(RB, LX, RC, LB)
    prm = I.noninteracting(_prm(dt=0.005, seed=4))
    g = np.random.default_rng(6)
    n = 400
    # start on the bridge and the connectors, where junctions are close
    ph = g.random(n) * 2 * math.pi
    x = np.column_stack([g.uniform(-LB / 2, LB / 2, n), RB * np.cos(ph), RB * np.sin(ph)])
    s = orc.System(surf, prm, n)
    s.set_state(x, I.maxwell(n, 1.0, 1.0, g))
    xs = [x]
    for _ in range(8):
        s.step(100)
        res = s.residual()
        # each position half solves g = 0 on the piece selected where the step
        # started; a particle that ends the step just across a junction is
        # measured on the next piece, which leaves the first one's extension
        # only at second order: |g|/|grad g| ~ (step length)^2 / R <~ 1e-5
        assert res["max_g_over_gradg"] < 1e-5
        xs.append(s.state()["x"])
    end = xs[-1]
    # some particles have left the bridge for the connectors or the face planes
    assert np.sum(np.abs(end[:, 0]) > LB / 2) > 20
