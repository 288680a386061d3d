"""Host-side logic of bench.py: the clock record keeps only the samples taken
inside the timed window and reports throttle reasons seen there."""
import datetime
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import bench  # noqa: E402


def _row(t, mhz, reasons=("Not Active",) * 4):
    return (f"{t.strftime('%Y/%m/%d %H:%M:%S.%f')[:-3]}, 0, {mhz}, 2070, 900.5, 0x0, "
            + ", ".join(reasons))


def test_clock_samples_outside_the_window_are_dropped():
    t = datetime.datetime(2026, 1, 2, 3, 4, 5)
    ms = datetime.timedelta(milliseconds=200)
    rows = [_row(t, 1000), _row(t + ms, 2070), _row(t + 2 * ms, 2070),
            _row(t + 3 * ms, 1900, ("Not Active", "Not Active", "Not Active", "Active")),
            _row(t + 5 * ms, 500, ("Active", "Not Active", "Not Active", "Not Active"))]
    out = bench.ClockSampler.parse("\n".join(rows), t + ms / 2, t + 3 * ms + ms / 2)
    assert out["samples"] == 3
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]
    assert abs(out["window_s"] - 0.6) < 1e-9


def test_no_sample_in_the_window_gives_none():
    t = datetime.datetime(2026, 1, 2, 3, 4, 5)
    assert bench.ClockSampler.parse(_row(t, 2070), t + datetime.timedelta(seconds=1),
                                    t + datetime.timedelta(seconds=2)) is None
    assert bench.ClockSampler.parse("garbage line\n", None, None) is None


def test_reference_arm_prints_one_json_line():
    """bench.py --impl reference runs the oracle on the host and prints the
    line the driver reads (small workload: the 1,000-particle sphere)."""
    import json
    import subprocess

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--workload",
                        "plain_sphere", "--steps", "2", "--warmup", "1"], capture_output=True, text=True,
                       timeout=600, cwd=root)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["steps"] == 2
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["cpu_baseline"]["cores"] >= 1 and line["config"]["engine"] == "global"
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
    assert line["config"]["workload"].startswith("plain_sphere")


def test_neighbour_list_defaults_and_cell_edge():
    """Per-workload Verlet-list defaults, explicit skins, and the cell edge
    the list needs (largest cutoff + skin)."""
    import numpy as np

    args = bench.parse(["--workload", "ellipsoid_torus"])
    assert bench.workload_skin(args) == 0.4 and bench.workload_max_neighbors(args) == 64
    args = bench.parse(["--workload", "bead_molecules"])
    assert bench.workload_max_neighbors(args) == 128
    args = bench.parse(["--workload", "capsids"])
    assert bench.workload_skin(args) == 0.4 and bench.workload_max_neighbors(args) == 256
    args = bench.parse(["--workload", "nve_surfaces"])  # the energy study keeps the cell list
    assert bench.workload_skin(args) == 0.0
    args = bench.parse(["--workload", "replicas", "--engine", "resident"])  # its own cell lists
    assert bench.workload_skin(args) == 0.0
    args = bench.parse(["--workload", "ellipsoid_torus", "--skin", "0", "--max-neighbors", "32"])
    assert bench.workload_skin(args) == 0.0 and bench.workload_max_neighbors(args) == 32
    rc = np.array([[1.12, 2.5], [2.5, 1.12]])
    systems = [{"params": {"rcut": rc, "cell_size": 0.0}}]
    assert bench.cells_for_skin(systems, 0.3)[0]["params"]["cell_size"] == 2.8
    systems = [{"params": {"rcut": rc, "cell_size": 0.0}}]
    assert bench.cells_for_skin(systems, 0.0)[0]["params"]["cell_size"] == 0.0


def test_algorithmic_bytes_per_particle():
    """The integrator and the pair kernel count the per-particle algorithmic
    bytes (each datum the method needs read or written once: 116 and 36 B in
    mixed precision, 128 and 68 B in float64) in both step forms; with the neighbour list the rebuild
    kernels count no bytes per step; the implementation's own bytes are
    reported beside them."""
    assert bench.algorithmic_bytes("integrate", 1000, 4096, "mixed", nlist=True) == 116_000
    assert bench.algorithmic_bytes("integrate", 1000, 4096, "mixed") == 116_000
    assert bench.algorithmic_bytes("pair", 1000, 4096, "mixed", nlist=True) == 36_000
    assert bench.algorithmic_bytes("integrate", 1000, 4096, "fp64") == 128_000
    assert bench.algorithmic_bytes("scan", 1000, 4096, "mixed", nlist=True) == 0
    assert bench.algorithmic_bytes("scan", 1000, 4096, "mixed") == 12 * 4096 + 16
    assert bench.impl_bytes("integrate", 1000, "mixed", True) > bench.algorithmic_bytes("integrate", 1000, 0,
                                                                                         "mixed")


def test_roofline_recomputes_from_kernel_times_bytes_and_peaks():
    """roofline.frac = (algorithmic bytes per particle x particles) / dominant
    kernel's duration / measured HBM peak; the float64-pipe fraction uses the
    measured FMA rate."""
    prof = {"pair": 0.020, "integrate": 0.030, "scan": 0.006}
    counts = {"integrate": {"fp64_inst": 2.5e6, "dram_bytes": 3e7}}
    r = bench.rooflines(prof, 250_000, 1 << 20, "mixed", 6766.7, counts, {"fp64": 6.0e11, "fp32": 4.0e13},
                        nlist=True)
    assert r["kernel"] == "integrate" and r["bound"] == "hbm"
    achieved = 116 * 250_000 / 30e-6 / 1e9
    assert abs(r["achieved"] - achieved) < 1e-9 and abs(r["frac"] - achieved / 6766.7) < 1e-12
    assert abs(r["fp64_pipe_frac"] - 2.5e6 / 30e-6 / 6.0e11) < 1e-12
    assert r["traffic"] == 3e7 and r["bytes_per_unit"] == 116 and r["units_per_launch"] == 250_000


def test_cpu_info_reports_cores():
    info = bench.cpu_info()
    assert info["cores"] >= 1


def test_list_autotuner_candidate_systems_leave_the_inputs_alone():
    """tune._with_cell_size gives copies of the system dicts whose cell edge is
    the largest cutoff + skin (the cell size a handle with that skin needs);
    the caller's dicts keep their parameters."""
    from paper_1411_3019_gb300 import inputs as I
    from paper_1411_3019_gb300 import tune

    systems = I.c5_bead_molecules(nmol=20, beads=5, R=6.0, seed=2)
    before = [dict(s["params"]) for s in systems]
    out = tune._with_cell_size(systems, 0.4)
    assert [s["params"]["cell_size"] for s in out] == [2.5 + 0.4] * len(systems)  # r_c = 2.5 between type-3 beads
    assert all(o is not s and o["params"] is not s["params"] for o, s in zip(out, systems))
    assert [s["params"]["cell_size"] for s in systems] == [b["cell_size"] for b in before]
    assert tune.LIST_SKINS == (0.3, 0.4, 0.5, 0.6) and tune.LIST_WARPS == (32, 16)
