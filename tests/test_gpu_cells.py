"""The cell list (index work of the pair step) against a host recomputation
from its definition, bit for bit: every particle's cell id, its bucket, the
bucket ranges and the canonical order (ascending particle id inside a
bucket)."""
import numpy as np
import pytest

from paper_1411_3019_gb300 import inputs as I
from paper_1411_3019_gb300 import md

pytestmark = pytest.mark.gpu


def _expected(h, systems, x):
    n = x.shape[0]
    cells = np.zeros(n, np.uint64)
    off = 0
    hashed = 0
    for s, sy in enumerate(systems):
        gi = md.md_grid_info(h, s)
        hashed = gi["hashed"]
        prm = sy["params"]
        xs = x[off:off + sy["n"]]
        c = np.zeros((sy["n"], 3), np.int64)
        mixed = prm["precision"] in ("mixed", 1)
        for d in range(3):
            if mixed:  # float32 binning with round-to-nearest operations
                f32 = np.float32
                v = xs[:, d].astype(f32)
                if prm["periodic"][d]:
                    lo = f32(prm["box_lo"][d])
                    L = f32(prm["box_hi"][d] - prm["box_lo"][d])
                    r = (v - lo).astype(f32)
                    v = (lo + (r - (L * np.floor(r / L)).astype(f32)).astype(f32)).astype(f32)
                t = ((v - f32(gi["lo"][d])).astype(f32) * f32(1.0 / gi["cs"][d])).astype(f32)
            else:
                v = xs[:, d].copy()
                if prm["periodic"][d]:
                    lo, L = prm["box_lo"][d], prm["box_hi"][d] - prm["box_lo"][d]
                    r = v - lo
                    v = lo + (r - L * np.floor(r / L))
                t = (v - gi["lo"][d]) * (1.0 / gi["cs"][d])
            c[:, d] = np.clip(np.floor(t), 0, gi["nc"][d] - 1)
        nc = gi["nc"].astype(np.int64)
        cells[off:off + sy["n"]] = gi["base"] + c[:, 0] + nc[0] * (c[:, 1] + nc[1] * c[:, 2])
        off += sy["n"]
    cells = cells.astype(np.uint32)
    if hashed:
        h32 = ((cells >> np.uint32(3)).astype(np.uint64) * 0x9E3779B1) & 0xFFFFFFFF
        bucket = ((h32 >> (35 - hashed)) << 3) | (cells & 7)
    else:
        bucket = cells.astype(np.uint64)
    return cells, bucket.astype(np.int64)


@pytest.mark.parametrize("case", ["dense_sphere", "hashed_batch", "periodic_crowders"])
def test_cell_list_is_the_definition(case):
    if case == "dense_sphere":
        systems = [I.sphere_system(n=1000, R=10.0, seed=1, dmin=0.8, precision="fp64")]
    elif case == "hashed_batch":
        # sparse particles on large surfaces: a grid of ~10^8 cells, so buckets are hashed
        systems = [I.sphere_system(n=3000, R=150.0, seed=3, dmin=1.0, precision="mixed", replica=0),
                   I.sphere_system(n=1000, R=60.0, seed=4, dmin=1.0, precision="mixed", replica=1)]
    else:
        systems = I.c3_bump_crowders(n_surf=500, n_free=1200, seed=6)
    sim = md.Simulation(systems)
    sim.set_state()
    for nsteps in (0, 7):
        sim.step(nsteps)
        sim.sync()
        x = sim.state()["x"]
        cl = md.md_cell_list(sim.h)
        cells, bucket = _expected(sim.h, systems, x)
        nb = cl["bucket_start"].shape[0] - 1
        order = np.lexsort((np.arange(x.shape[0]), bucket))
        assert np.array_equal(cl["sorted_ids"], order.astype(np.uint32))
        assert np.array_equal(cl["sorted_cells"], cells[order])
        counts = np.bincount(bucket, minlength=nb)
        start = np.concatenate([[0], np.cumsum(counts)]).astype(np.uint32)
        assert np.array_equal(cl["bucket_start"], start)
    if case == "dense_sphere":
        assert md.md_grid_info(sim.h, 0)["hashed"] == 0
    if case == "hashed_batch":
        assert md.md_grid_info(sim.h, 0)["hashed"] > 0
    sim.close()
