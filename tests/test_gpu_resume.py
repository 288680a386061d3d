"""Reproducibility: two runs give the same bits; a checkpoint (x^k,
p^{k-1/2}, k) restored into a new handle repeats the uninterrupted
trajectory bit for bit (the noise is a pure function of seed, replica,
particle and step); torch device memory and streams drive the same path."""
import numpy as np
import pytest

from paper_1411_3019_gb300 import inputs as I
from paper_1411_3019_gb300 import md

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_runs_are_bitwise_repeatable_and_resumable(precision):
    systems = I.c2_ellipsoid_torus(n_ell=4000, n_tor=1500, seed=8, precision=precision)
    with md.Simulation(systems) as a:
        a.set_state()
        a.step(30)
        ck = a.state()
        a.step(30)
        xa = a.state()
    with md.Simulation(systems) as b:
        b.set_state()
        b.step(60)
        xb = b.state()
    assert np.array_equal(xa["x"], xb["x"]) and np.array_equal(xa["v"], xb["v"])
    with md.Simulation(systems) as c:
        c.set_state()
        md.md_restore(c.h, ck["x"], ck["p_half"], ck["step"])
        c.step(30)
        xc = c.state()
    assert xc["step"] == 60
    assert np.array_equal(xa["x"], xc["x"])
    assert np.array_equal(xa["p_half"], xc["p_half"])


def test_torch_device_buffers_and_stream():
    torch = pytest.importorskip("torch")
    systems = [I.sphere_system(n=500, R=9.0, seed=4, dmin=0.9, precision="mixed")]
    s = systems[0]
    with md.Simulation(systems) as ref:
        ref.set_state()
        ref.step(20)
        want = ref.state()
    dev = torch.device("cuda:0")
    x = torch.tensor(s["x"], dtype=torch.float64, device=dev)
    v = torch.tensor(s["v"], dtype=torch.float64, device=dev)
    stream = torch.cuda.Stream()
    with md.Simulation(systems, stream=stream) as sim:
        md.md_set_state_device(sim.h, x, v)
        sim.step(20)
        out_x = torch.empty_like(x)
        out_v = torch.empty_like(v)
        md.md_get_state_device(sim.h, out_x, out_v)
        stream.synchronize()
        assert np.array_equal(out_x.cpu().numpy(), want["x"])
        assert np.array_equal(out_v.cpu().numpy(), want["v"])
