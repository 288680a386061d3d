"""The C-ABI library without a GPU: it builds, loads, exports every entry
point include/md.h declares, its structs have the layout the binding
assumes, and argument errors come back before any device work."""
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "md.h")


@pytest.fixture(scope="module")
def md():
    from paper_1411_3019_gb300 import _build, md
    _build.build()
    md.lib()
    return md


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(md_[a-z_]+)\s*\(", text)))


def test_library_exports_every_declared_entry_point(md):
    names = _declared()
    assert "md_step" in names and "md_create_batch" in names
    out = subprocess.run(["nm", "-D", "--defined-only", md.library_path()], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r" T (md_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        assert hasattr(md.lib(), n)


def test_struct_layout_matches_the_header(md, tmp_path):
    probe = tmp_path / "probe.c"
    fields = {"md_surface": [f for f, _ in md.md_surface._fields_],
              "md_params": [f for f, _ in md.md_params._fields_],
              "md_obs": [f for f, _ in md.md_obs._fields_]}
    lines = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{HEADER}"', "int main(void){"]
    for st, fs in fields.items():
        lines.append(f'printf("{st} %zu\\n", sizeof({st}));')
        for f in fs:
            lines.append(f'printf("{st}.{f} %zu\\n", offsetof({st}, {f}));')
    lines.append("return 0;}")
    probe.write_text("\n".join(lines))
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-std=c11", "-o", str(exe), str(probe)], check=True)
    got = dict(line.split() for line in subprocess.run([str(exe)], capture_output=True, text=True,
                                                        check=True).stdout.splitlines())
    for st in fields:
        cls = getattr(md, st)
        assert int(got[st]) == __import__("ctypes").sizeof(cls), st
        for f in fields[st]:
            assert int(got[f"{st}.{f}"]) == getattr(cls, f).offset, (st, f)


def _valid():
    from paper_1411_3019_gb300 import inputs
    return inputs.sphere_system(n=10, R=3.0, seed=1, dmin=0.9)


@pytest.mark.parametrize("change", [
    ("params", "dt", 0.0), ("params", "dt", -1.0), ("params", "rattle_tol", 0.0),
    ("params", "precision", 7), ("params", "ntypes", 0), ("params", "ntypes", 9),
    ("params", "gamma", -1.0), ("params", "max_newton", -1),
    ("surface", "p", (-1.0, 0, 0, 0)), ("surface", "kind", 42), ("params", "pair_form", 2),
])
def test_bad_arguments_are_rejected_on_the_host(md, change):
    s = _valid()
    where, key, val = change
    s[where] = dict(s[where])
    s[where][key] = val
    with pytest.raises(md.MdError) as e:
        md.md_create(s["surface"], s["params"], s["n"])
    assert e.value.code == md.MD_ERR_INVALID_ARG
    assert md.md_last_error(None)


def test_asymmetric_tables_and_bad_geometry_are_rejected(md):
    s = _valid()
    prm = dict(s["params"], ntypes=2, eps=np.array([[1.0, 1.0], [0.5, 1.0]]),
               sigma=np.ones((2, 2)), rcut=np.ones((2, 2)))
    with pytest.raises(md.MdError):
        md.md_create(s["surface"], prm, 10)
    bump = {"kind": "gaussian_bump", "center": (0, 0, 0), "p": (5.0, 3.0, 0, 0)}
    with pytest.raises(md.MdError):  # a bump needs periodic x, y
        md.md_create(bump, s["params"], 10)
    prm = dict(s["params"], box_lo=(0, 0, 0), box_hi=(2.0, 2.0, 2.0), periodic=(1, 1, 1))
    with pytest.raises(md.MdError):  # fewer than 3 cells on a periodic axis
        md.md_create({"kind": "none"}, prm, 10)
    with pytest.raises(md.MdError):  # a free system needs a box for its grid
        md.md_create({"kind": "none"}, s["params"], 10)


def test_batch_must_share_interactions(md):
    a, b = _valid(), _valid()
    b["params"] = dict(b["params"], precision="fp64" if a["params"]["precision"] == "mixed" else "mixed")
    with pytest.raises(md.MdError):
        md.md_create_batch([a["surface"], b["surface"]], [a["params"], b["params"]], [10, 10])


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    from paper_1411_3019_gb300 import md as mdmod
    monkeypatch.setattr(mdmod, "_lib", None)
    monkeypatch.setattr(mdmod, "library_path", lambda: str(tmp_path / "nope.so"))
    with pytest.raises(RuntimeError, match="missing"):
        mdmod.lib()


def test_binding_constants_match_the_header():
    """Every status code, flag, option, pair form and wall kind the header
    defines has the same value in the binding, and so do the surface kinds
    and precisions."""
    from paper_1411_3019_gb300 import md as binding

    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    defines = {k: int(v.rstrip("uU"), 0) for k, v in
               re.findall(r"#define\s+(MD_[A-Z0-9_]+)\s+(0x[0-9a-fA-F]+u?|\d+)\b", text)}
    wanted = [k for k in defines if k.startswith(("MD_OK", "MD_ERR_", "MD_FLAG_", "MD_OPT_", "MD_PAIR_", "MD_WALL_"))]
    assert len(wanted) >= 24
    for k in wanted:
        assert getattr(binding, k) == defines[k], k
    kinds = dict(re.findall(r"\bMD_SURF_([A-Z0-9_]+)\s*=\s*(\d+)", text))
    assert {k.lower(): int(v) for k, v in kinds.items()} == binding.SURF_KINDS
    assert binding.PRECISION == {"fp64": defines["MD_PREC_FP64"], "mixed": defines["MD_PREC_MIXED"]}
