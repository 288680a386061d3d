"""The oracle's OpenMP threads only split its independent per-particle
loops: the state after several steps is the same bit for bit at any thread
count (the CPU baseline and the reference arm run it on every core)."""
import numpy as np

from paper_1411_3019_gb300 import inputs as I


def test_thread_count_changes_no_bit(orc):
    sy = I.c2_ellipsoid_torus(n_ell=6000, n_tor=1500, seed=4)[0]
    out = {}
    for k in (1, 3):
        assert orc.set_threads(k) in (1, k)  # 1 where the oracle was built without OpenMP
        o = orc.System(sy["surface"], sy["params"], sy["n"], force_mode="cells")
        o.set_state(sy["x"], sy["v"], sy["type"], None, sy["constrained"])
        o.step(4)
        out[k] = o.state()
    orc.set_threads(1)
    for key in ("x", "v", "p_half"):
        assert np.array_equal(out[1][key], out[3][key]), key
