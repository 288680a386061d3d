"""Pins of the oracle's random numbers: Philox4x32-10 against the published
known-answer vectors, the Box-Muller normals against the normal law, and the
tangent-plane projection of isotropic noise (Section 3.1: projecting the
random force on the tangent plane leaves a 2-D normal)."""
import os

import numpy as np
import pytest
from scipy import stats

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat_rows():
    rows = []
    with open(GOLDEN) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            w = [int(t, 16) for t in line.split()]
            rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,expect", _kat_rows())
def test_philox_known_answers(orc, ctr, key, expect):
    out = orc.philox4x32_10(ctr, key)
    assert [int(v) for v in out] == expect


def _draws(orc, n, seed=7, replica=3, step=11):
    return np.array([orc.gauss3(seed, replica, i, step) for i in range(n)])


def test_normals_moments_and_ks(orc):
    z = _draws(orc, 20000)
    for c in range(3):
        col = z[:, c]
        assert abs(col.mean()) < 4 / np.sqrt(col.size)
        assert abs(col.var() - 1.0) < 4 * np.sqrt(2.0 / col.size)
        assert stats.kstest(col, "norm").pvalue > 1e-3
    corr = np.corrcoef(z.T)
    assert np.all(np.abs(corr - np.eye(3)) < 4 / np.sqrt(z.shape[0]))


def test_normals_depend_on_every_key_and_counter_word(orc):
    base = orc.gauss3(1, 0, 5, 100)
    for args in [(2, 0, 5, 100), (1, 1, 5, 100), (1, 0, 6, 100), (1, 0, 5, 101),
                 (1, 0, 5, 100 + (1 << 32)), (1 + (1 << 32), 0, 5, 100)]:
        other = orc.gauss3(*args)
        if args[0] == 1 + (1 << 32):
            # only the low 32 bits of the seed are a key word
            assert np.array_equal(other, base)
        else:
            assert not np.allclose(other, base)


def test_normals_are_box_muller_of_the_philox_words(orc):
    """The three normals are the Box-Muller pair of words (0, 1) and the
    cosine branch of words (2, 3), with u = ((w >> 9) + 1/2) 2^-23."""
    seed, rep, pid, step = 12345, 9, 77, (3 << 32) + 5
    w = orc.philox4x32_10([pid, step & 0xFFFFFFFF, step >> 32, 0], [seed & 0xFFFFFFFF, rep])
    u = ((w >> 9).astype(np.float64) + 0.5) / 2.0 ** 23
    expect = [np.sqrt(-2 * np.log(u[0])) * np.cos(2 * np.pi * u[1]),
              np.sqrt(-2 * np.log(u[0])) * np.sin(2 * np.pi * u[1]),
              np.sqrt(-2 * np.log(u[2])) * np.cos(2 * np.pi * u[3])]
    np.testing.assert_allclose(orc.gauss3(seed, rep, pid, step), expect, rtol=1e-14, atol=1e-15)


def test_tangent_projection_stays_gaussian(orc):
    z = _draws(orc, 20000, seed=3)
    rng = np.random.default_rng(0)
    nrm = rng.standard_normal(3)
    nrm /= np.linalg.norm(nrm)
    t1 = np.cross(nrm, [1.0, 0.0, 0.0])
    t1 /= np.linalg.norm(t1)
    t2 = np.cross(nrm, t1)
    proj = z - np.outer(z @ nrm, nrm)
    for t in (t1, t2):
        comp = proj @ t
        assert stats.kstest(comp, "norm").pvalue > 1e-3
    assert np.max(np.abs(proj @ nrm)) < 1e-12
