"""md_forces_noalloc: forces of one system without any device allocation,
for callers that cannot allocate device memory where they need forces: an
application whose device memory all belongs to its own pool allocator, or a
caller on a latency-critical path that must not wait on the driver's
allocator. The entry point works in the library's fixed scratch array. Its
forces must match md_forces of a handle with the same system (within the
force tolerance: its cell grid may differ, so float32 sums can differ in the
last bits) and the oracle, on two calls in a row and after a call on a
larger, differently laid out system (the array keeps the previous call's
contents, which must not leak into the next), and the device's free memory
must not change across a call (after the first call on the device, which
loads the library's device code and its scratch array)."""
import numpy as np
import pytest

from paper_1411_3019_gb300 import inputs as I
from paper_1411_3019_gb300 import md

from parity_util import FORCE_REL, assert_forces

pytestmark = pytest.mark.gpu


def _cases():
    return [
        ("sphere_fp64", [I.sphere_system(n=1000, R=10.0, seed=1, dmin=0.8, precision="fp64", dt=0.001,
                                         tol=1e-12)]),
        ("bead_molecules_mixed", I.c5_bead_molecules(nmol=300, beads=5, R=10.0, seed=4, precision="mixed")),
        ("sparse_sphere_hashed_mixed", [I.sphere_system(n=3000, R=150.0, seed=3, dmin=1.0,
                                                        precision="mixed")]),
        ("plane2d_mixed", I.sphere_and_plane2d(n=2000, seed=5, precision="mixed")[1]),
    ]


def _rel(f, ref):
    return float(np.max(np.linalg.norm(f - ref, axis=1) / np.maximum(np.linalg.norm(ref, axis=1), 1.0)))


def _reference(systems):
    """Positions after a few steps and md_forces at them."""
    with md.Simulation(systems) as sim:
        sim.set_state()
        sim.step(5)
        sim.sync()
        x = sim.state()["x"]
        f, u = sim.forces()
    return x, f, u


def _load(torch):
    """One small call first: the first call on a device loads the library's
    device code with its scratch array (set-up, not an allocation of the
    call), so the free-memory checks below measure warm calls."""
    sy = I.sphere_system(n=10, R=3.0, seed=1, dmin=0.9)
    d_x = torch.tensor(sy["x"], dtype=torch.float64, device="cuda:0")
    d_f = torch.empty((10, 3), dtype=torch.float64, device="cuda:0")
    md.md_forces_noalloc(sy["surface"], sy["params"], 10, d_x, d_f)


def _noalloc(torch, sy, x):
    dev = torch.device("cuda:0")
    d_x = torch.tensor(x, dtype=torch.float64, device=dev)
    d_type = torch.tensor(sy["type"], dtype=torch.int32, device=dev)
    d_con = torch.tensor(sy["constrained"], dtype=torch.uint8, device=dev)
    d_f = torch.full((sy["n"], 3), float("nan"), dtype=torch.float64, device=dev)
    d_u = torch.full((sy["n"],), float("nan"), dtype=torch.float64, device=dev)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    md.md_forces_noalloc(sy["surface"], sy["params"], sy["n"], d_x, d_f, d_type=d_type, d_con=d_con, d_u=d_u)
    free1 = torch.cuda.mem_get_info()[0]
    return d_f.cpu().numpy(), d_u.cpu().numpy(), free0 - free1


@pytest.mark.parametrize("name,systems", _cases(), ids=[c[0] for c in _cases()])
def test_noalloc_forces_match_md_forces_and_the_oracle_on_two_calls(name, systems):
    torch = pytest.importorskip("torch")
    sy = systems[0]
    precision = "fp64" if sy["params"]["precision"] == "fp64" else "mixed"
    x, f_ref, u_ref = _reference(systems)
    _load(torch)
    outs = []
    for _ in range(2):
        f, u, grown = _noalloc(torch, sy, x)
        assert grown == 0  # the call allocated no device memory
        assert np.all(np.isfinite(f)) and np.all(np.isfinite(u))
        assert _rel(f, f_ref) <= FORCE_REL[precision]
        assert_forces(systems, x, f, precision)
        np.testing.assert_allclose(u.sum(), u_ref.sum(), rtol=max(FORCE_REL[precision], 1e-10))
        outs.append(f)
    assert np.array_equal(outs[0], outs[1])


def test_noalloc_after_a_larger_hashed_system():
    """A sparse 3,000-particle sphere (hashed buckets) and then a dense
    1,000-particle sphere (buckets = cells): each call matches md_forces of
    its own system, so nothing of the first call's scratch leaks into the
    second."""
    torch = pytest.importorskip("torch")
    first = [I.sphere_system(n=3000, R=150.0, seed=3, dmin=1.0, precision="mixed")]
    second = [I.sphere_system(n=1000, R=10.0, seed=1, dmin=0.8, precision="mixed", dt=0.001)]
    _load(torch)
    for systems in (first, second):
        x, f_ref, _ = _reference(systems)
        f, _, grown = _noalloc(torch, systems[0], x)
        assert grown == 0
        assert _rel(f, f_ref) <= FORCE_REL["mixed"]
        assert_forces(systems, x, f, "mixed")


def test_noalloc_rejects_systems_beyond_its_limit():
    torch = pytest.importorskip("torch")
    sy = I.sphere_system(n=10, R=3.0, seed=1, dmin=0.9)
    d = torch.zeros((70000, 3), dtype=torch.float64, device="cuda:0")
    with pytest.raises(md.MdError) as e:
        md.md_forces_noalloc(sy["surface"], sy["params"], 70000, d, d)
    assert e.value.code == md.MD_ERR_INVALID_ARG
    assert "65536" in md.md_last_error(None)


def test_noalloc_rejects_a_type_outside_ntypes():
    """A type equal to ntypes is reported as a bad input, and the next call
    with valid types still matches md_forces."""
    torch = pytest.importorskip("torch")
    systems = [I.sphere_system(n=1000, R=10.0, seed=1, dmin=0.8, precision="mixed", dt=0.001)]
    sy = dict(systems[0])
    x, f_ref, _ = _reference(systems)
    _load(torch)
    bad = dict(sy, type=np.asarray(sy["type"]).copy())
    bad["type"][7] = sy["params"]["ntypes"]
    with pytest.raises(md.MdError) as e:
        _noalloc(torch, bad, x)
    assert e.value.code == md.MD_ERR_INVALID_ARG
    f, _, _ = _noalloc(torch, sy, x)
    assert _rel(f, f_ref) <= FORCE_REL["mixed"]


@pytest.mark.parametrize("mode", ["relaxed", "thread_local"])
def test_noalloc_while_another_thread_captures_a_graph(mode):
    """Thread A captures a small torch graph (relaxed or thread-local capture
    mode) and holds the capture open while this thread calls
    md_forces_noalloc on a non-blocking stream: the call runs, its forces
    equal md_forces', and A's capture completes and replays."""
    import threading

    torch = pytest.importorskip("torch")
    systems = [I.sphere_system(n=1000, R=10.0, seed=1, dmin=0.8, precision="mixed", dt=0.001)]
    sy = systems[0]
    x, f_ref, _ = _reference(systems)
    _load(torch)
    dev = torch.device("cuda:0")
    d_x = torch.tensor(x, dtype=torch.float64, device=dev)
    d_type = torch.tensor(sy["type"], dtype=torch.int32, device=dev)
    d_con = torch.tensor(sy["constrained"], dtype=torch.uint8, device=dev)
    d_f = torch.zeros((sy["n"], 3), dtype=torch.float64, device=dev)
    a = torch.zeros(1 << 20, device=dev)
    s_cap, s_b = torch.cuda.Stream(), torch.cuda.Stream()  # torch streams are non-blocking
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    started, release, errors = threading.Event(), threading.Event(), []

    def capture():
        try:
            with torch.cuda.stream(s_cap):
                g.capture_begin(capture_error_mode=mode)
                a.add_(1.0)
                started.set()
                release.wait(timeout=30)
                a.mul_(2.0)
                g.capture_end()
        except Exception as e:  # reported below
            errors.append(e)
            started.set()

    t = threading.Thread(target=capture)
    t.start()
    assert started.wait(30)
    try:
        md.md_forces_noalloc(sy["surface"], sy["params"], sy["n"], d_x, d_f, d_type=d_type, d_con=d_con,
                             stream=s_b)
    finally:
        release.set()
        t.join()
    assert not errors, errors
    g.replay()
    torch.cuda.synchronize()
    assert float(a[0]) == 2.0
    assert _rel(d_f.cpu().numpy(), f_ref) <= FORCE_REL["mixed"]
