"""md_forces_noalloc: forces without any device allocation, for callers that
cannot allocate device memory where they need forces (for example a thread
working while a CUDA graph is captured in global mode, or an application whose
device memory belongs to its own allocator). The entry point uses the
library's fixed scratch array; its result must match md_forces of a handle
with the same system, on two calls in a row (the array keeps the previous
call's contents, which must not leak into the next)."""
import numpy as np
import pytest

from paper_1411_3019_gb300 import inputs as I
from paper_1411_3019_gb300 import md

from parity_util import FORCE_REL

pytestmark = pytest.mark.gpu


def _cases():
    return [
        ("sphere_fp64", [I.sphere_system(n=1000, R=10.0, seed=1, dmin=0.8, precision="fp64", dt=0.001,
                                         tol=1e-12)]),
        ("bead_molecules_mixed", I.c5_bead_molecules(nmol=300, beads=5, R=10.0, seed=4, precision="mixed")),
        ("sparse_sphere_hashed_mixed", [I.sphere_system(n=3000, R=150.0, seed=3, dmin=1.0,
                                                        precision="mixed")]),
    ]


def _rel(f, ref):
    return float(np.max(np.linalg.norm(f - ref, axis=1) / np.maximum(np.linalg.norm(ref, axis=1), 1.0)))


@pytest.mark.parametrize("name,systems", _cases(), ids=[c[0] for c in _cases()])
def test_noalloc_forces_match_md_forces_on_two_calls(name, systems):
    torch = pytest.importorskip("torch")
    sy = systems[0]
    with md.Simulation(systems) as sim:
        sim.set_state()
        sim.step(5)
        sim.sync()
        x = sim.state()["x"]
        f_ref, u_ref = sim.forces()
    dev = torch.device("cuda:0")
    d_x = torch.tensor(x, dtype=torch.float64, device=dev)
    d_type = torch.tensor(sy["type"], dtype=torch.int32, device=dev)
    d_con = torch.tensor(sy["constrained"], dtype=torch.uint8, device=dev)
    tol = FORCE_REL["fp64" if sy["params"]["precision"] == "fp64" else "mixed"]
    outs = []
    for _ in range(2):
        d_f = torch.full((sy["n"], 3), float("nan"), dtype=torch.float64, device=dev)
        d_u = torch.full((sy["n"],), float("nan"), dtype=torch.float64, device=dev)
        md.md_forces_noalloc(sy["surface"], sy["params"], sy["n"], d_x, d_f, d_type=d_type, d_con=d_con,
                             d_u=d_u)
        f, u = d_f.cpu().numpy(), d_u.cpu().numpy()
        assert np.all(np.isfinite(f)) and np.all(np.isfinite(u))
        assert _rel(f, f_ref) <= tol
        np.testing.assert_allclose(u.sum(), u_ref.sum(), rtol=max(tol, 1e-10))
        outs.append(f)
    assert np.array_equal(outs[0], outs[1])


def test_noalloc_rejects_systems_beyond_its_limit():
    torch = pytest.importorskip("torch")
    sy = I.sphere_system(n=10, R=3.0, seed=1, dmin=0.9)
    d = torch.zeros((70000, 3), dtype=torch.float64, device="cuda:0")
    with pytest.raises(md.MdError) as e:
        md.md_forces_noalloc(sy["surface"], sy["params"], 70000, d, d)
    assert e.value.code == md.MD_ERR_INVALID_ARG
    assert "65536" in md.md_last_error(None)
