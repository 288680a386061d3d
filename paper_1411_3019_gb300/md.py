"""Thin ctypes binding of libsurfmd.so, the C ABI declared in include/md.h.

The functions carry the C names (md_create, md_set_state, md_step, ...) and
only marshal arguments: every step of the method runs in the CUDA kernels of
the library. There is no CPU fallback: if the library is missing the first
call raises.

Inputs are numpy arrays ([n, 3] float64 positions/velocities) or, for the
*_device variants, CUDA device pointers (ints, or objects with data_ptr()
such as torch tensors).
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import _build

MAX_TYPES = 8
SURF_KINDS = {"none": 0, "plane": 1, "sphere": 2, "ellipsoid": 3, "torus": 4, "gaussian_bump": 5,
              "cylinder": 6, "xy2d": 7, "thylakoid": 8}
PRECISION = {"fp64": 0, "mixed": 1}
MD_OK, MD_ERR_INVALID_ARG, MD_ERR_CUDA, MD_ERR_RATTLE_DIVERGED = 0, 1, 2, 3
MD_ERR_NONFINITE, MD_ERR_OUT_OF_GRID, MD_ERR_TIMEOUT, MD_ERR_NO_DEVICE = 4, 5, 6, 7
MD_ERR_NLIST_FULL = 8
MD_FLAG_RATTLE_DIVERGED, MD_FLAG_NONFINITE, MD_FLAG_OUT_OF_GRID, MD_FLAG_TIMEOUT = 1, 2, 4, 8
MD_OPT_PAIR_LANES = 1
MD_PAIR_TRUNC_SHIFT, MD_PAIR_LINEAR_SMOOTH = 0, 1
MD_WALL_PLANES, MD_WALL_SPHERE = 0, 1
MD_OPT_PAIR_ORDER = 2
MD_OPT_ENGINE = 3
MD_OPT_RESIDENT_THREADS = 4
MD_OPT_RESIDENT_STEPS = 5
MD_OPT_PAIR_TILE = 6
MD_OPT_NLIST_BUILDS = 7
MD_OPT_SPIN_LIMIT = 8
MD_OPT_PAIR_QUEUE = 9
MD_OPT_FUSED_REBUILD = 10
MD_OPT_LIST_WARP = 11
MD_OPT_STORE_NOISE = 12
ERROR_NAMES = {0: "MD_OK", 1: "MD_ERR_INVALID_ARG", 2: "MD_ERR_CUDA", 3: "MD_ERR_RATTLE_DIVERGED",
               4: "MD_ERR_NONFINITE", 5: "MD_ERR_OUT_OF_GRID", 6: "MD_ERR_TIMEOUT", 7: "MD_ERR_NO_DEVICE",
               8: "MD_ERR_NLIST_FULL"}


class MdError(RuntimeError):
    def __init__(self, code: int, message: str):
        super().__init__(f"{ERROR_NAMES.get(code, code)}: {message}")
        self.code = code
        self.message = message


class md_surface(C.Structure):
    _fields_ = [("kind", C.c_int32), ("reserved", C.c_int32), ("center", C.c_double * 3),
                ("p", C.c_double * 4)]


class md_params(C.Structure):
    _fields_ = [("dt", C.c_double), ("kT", C.c_double), ("gamma", C.c_double),
                ("rattle_tol", C.c_double), ("max_newton", C.c_int32), ("frozen_normal", C.c_int32),
                ("precision", C.c_int32), ("ntypes", C.c_int32),
                ("mass", C.c_double * MAX_TYPES),
                ("eps", (C.c_double * MAX_TYPES) * MAX_TYPES),
                ("sigma", (C.c_double * MAX_TYPES) * MAX_TYPES),
                ("rcut", (C.c_double * MAX_TYPES) * MAX_TYPES),
                ("box_lo", C.c_double * 3), ("box_hi", C.c_double * 3), ("periodic", C.c_int32 * 3),
                ("beads_per_mol", C.c_int32), ("bond_k", C.c_double), ("bond_r0", C.c_double),
                ("exclude_intramol", C.c_int32), ("wall_enable", C.c_int32),
                ("wall_lo_z", C.c_double), ("wall_hi_z", C.c_double), ("wall_eps", C.c_double),
                ("wall_sigma", C.c_double), ("seed", C.c_uint64), ("replica", C.c_uint32),
                ("pair_form", C.c_int32), ("cell_size", C.c_double),
                ("angle_k", C.c_double), ("angle_theta0", C.c_double), ("bond_r0_mix", C.c_int32),
                ("wall_kind", C.c_int32), ("wall_radius", C.c_double), ("wall_center", C.c_double * 3)]


class md_obs(C.Structure):
    _fields_ = [("step", C.c_uint64), ("n", C.c_int64), ("ndof", C.c_int64), ("kinetic", C.c_double),
                ("potential", C.c_double), ("kT", C.c_double), ("max_g_over_gradg", C.c_double),
                ("max_n_dot_v", C.c_double), ("msd", C.c_double), ("r0_dot_rt", C.c_double)]


_lib = None
_lock = threading.Lock()


def library_path() -> str:
    return _build.LIB


def lib():
    """The loaded CUDA library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            path = library_path()
            if not os.path.exists(path):
                raise RuntimeError(f"{path} is missing: build it with __graft_entry__.build()")
            L = C.CDLL(path)
            vp, i32, i64, u64, dp = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64, C.c_void_p
            sig = {
                "md_version": ([], C.c_int),
                "md_create": ([C.POINTER(md_surface), C.POINTER(md_params), i64, C.POINTER(vp)], C.c_int),
                "md_create_batch": ([i32, C.POINTER(md_surface), C.POINTER(md_params), C.POINTER(i64),
                                     C.POINTER(vp)], C.c_int),
                "md_set_stream": ([vp, vp], C.c_int),
                "md_set_state": ([vp, dp, dp, dp, dp, dp, u64], C.c_int),
                "md_set_state_device": ([vp, dp, dp, dp, dp, dp, u64], C.c_int),
                "md_restore": ([vp, dp, dp, u64], C.c_int),
                "md_step": ([vp, i64], C.c_int),
                "md_sync": ([vp], C.c_int),
                "md_status": ([vp, C.POINTER(C.c_uint32)], C.c_int),
                "md_get_state": ([vp, dp, dp, dp, C.POINTER(u64)], C.c_int),
                "md_get_state_device": ([vp, dp, dp, dp], C.c_int),
                "md_forces": ([vp, dp, dp], C.c_int),
                "md_constraint_residual": ([vp, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                            C.POINTER(C.c_double)], C.c_int),
                "md_observables": ([vp, C.POINTER(md_obs), i32, C.POINTER(i32)], C.c_int),
                "md_info": ([vp, C.POINTER(i64), C.POINTER(i32), C.POINTER(u64)], C.c_int),
                "md_last_launch_count": ([vp, C.POINTER(i64)], C.c_int),
                "md_grid_info": ([vp, i32, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                  C.POINTER(i32), C.POINTER(C.c_uint32), C.POINTER(i32)], C.c_int),
                "md_cell_list": ([vp, dp, dp, dp, C.POINTER(C.c_uint32)], C.c_int),
                "md_profile_step": ([vp, i64, C.POINTER(C.c_double), i32, C.POINTER(i32)], C.c_int),
                "md_profile_kernel_name": ([vp, i32], C.c_char_p),
                "md_forces_noalloc": ([C.POINTER(md_surface), C.POINTER(md_params), i64, dp, dp, dp, dp, dp,
                                       dp, vp], C.c_int),
                "md_set_option": ([vp, i32, i64], C.c_int),
                "md_set_neighbor_list": ([vp, C.c_double, i32], C.c_int),
                "md_check_conversions": ([vp, i64, vp, vp], C.c_int),
                "md_measure_fma_peak": ([i32, i32, C.POINTER(C.c_double)], C.c_int),
                "md_get_option": ([vp, i32, C.POINTER(i64)], C.c_int),
                "md_last_error": ([vp], C.c_char_p),
                "md_destroy": ([vp], None),
            }
            for name, (args, res) in sig.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = res
            _lib = L
    return _lib


def _check(h, rc: int):
    if rc != MD_OK:
        msg = lib().md_last_error(h)
        raise MdError(rc, msg.decode() if msg else "")


# ---------------------------------------------------------------------------
# dict -> struct
# ---------------------------------------------------------------------------
def make_surface(surf: dict | None) -> md_surface:
    s = md_surface()
    surf = surf or {"kind": "none"}
    kind = surf.get("kind", "none")
    s.kind = SURF_KINDS[kind] if isinstance(kind, str) else int(kind)
    for k, v in enumerate(surf.get("center", (0.0, 0.0, 0.0))):
        s.center[k] = float(v)
    for k, v in enumerate(surf.get("p", ())):
        s.p[k] = float(v)
    return s


def make_params(prm: dict) -> md_params:
    P = md_params()
    P.dt = prm["dt"]
    P.kT = prm.get("kT", 1.0)
    P.gamma = prm.get("gamma", 1.0)
    P.rattle_tol = prm.get("rattle_tol", 1e-10)
    P.max_newton = prm.get("max_newton", 30)
    P.frozen_normal = prm.get("frozen_normal", 0)
    prec = prm.get("precision", "mixed")
    P.precision = PRECISION[prec] if isinstance(prec, str) else int(prec)
    nt = prm.get("ntypes", 1)
    P.ntypes = nt
    mass = prm.get("mass", [1.0] * nt)
    for a in range(MAX_TYPES):
        P.mass[a] = float(mass[a]) if a < len(mass) else 1.0
    for key in ("eps", "sigma", "rcut"):
        tab = np.asarray(prm.get(key, np.zeros((nt, nt))), dtype=np.float64)
        arr = getattr(P, key)
        for a in range(tab.shape[0]):
            for b in range(tab.shape[1]):
                arr[a][b] = float(tab[a, b])
    for k in range(3):
        P.box_lo[k] = float(prm.get("box_lo", (0.0, 0.0, 0.0))[k])
        P.box_hi[k] = float(prm.get("box_hi", (0.0, 0.0, 0.0))[k])
        P.periodic[k] = int(prm.get("periodic", (0, 0, 0))[k])
    P.beads_per_mol = prm.get("beads_per_mol", 0)
    P.bond_k = prm.get("bond_k", 0.0)
    P.bond_r0 = prm.get("bond_r0", 0.0)
    P.exclude_intramol = prm.get("exclude_intramol", 0)
    P.wall_enable = prm.get("wall_enable", 0)
    P.wall_lo_z = prm.get("wall_lo_z", 0.0)
    P.wall_hi_z = prm.get("wall_hi_z", 0.0)
    P.wall_eps = prm.get("wall_eps", 1.0)
    P.wall_sigma = prm.get("wall_sigma", 1.0)
    P.seed = prm.get("seed", 1) & 0xFFFFFFFFFFFFFFFF
    P.replica = prm.get("replica", 0) & 0xFFFFFFFF
    P.pair_form = int(prm.get("pair_form", 0))
    P.cell_size = prm.get("cell_size", 0.0)
    P.angle_k = float(prm.get("angle_k", 0.0))
    P.angle_theta0 = float(prm.get("angle_theta0", 0.0))
    P.bond_r0_mix = int(prm.get("bond_r0_mix", 0))
    P.wall_kind = int(prm.get("wall_kind", 0))
    P.wall_radius = float(prm.get("wall_radius", 0.0))
    for k in range(3):
        P.wall_center[k] = float(prm.get("wall_center", (0.0, 0.0, 0.0))[k])
    return P


def _host(a, dtype, shape=None):
    if a is None:
        return None, None
    arr = np.ascontiguousarray(a, dtype=dtype)
    if shape is not None:
        arr = arr.reshape(shape)
    return arr, arr.ctypes.data_as(C.c_void_p)


def _dptr(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return C.c_void_p(a.data_ptr())
    return C.c_void_p(int(a))


# ---------------------------------------------------------------------------
# the C ABI, one Python function per entry point
# ---------------------------------------------------------------------------
def md_version() -> int:
    return lib().md_version()


def md_create(surface: dict | None, params: dict, n: int):
    h = C.c_void_p()
    S, P = make_surface(surface), make_params(params)
    rc = lib().md_create(C.byref(S), C.byref(P), int(n), C.byref(h))
    _check(None, rc)
    return h


def md_create_batch(surfaces, params_list, n_per_sys):
    ns = len(surfaces)
    S = (md_surface * ns)(*[make_surface(s) for s in surfaces])
    P = (md_params * ns)(*[make_params(p) for p in params_list])
    N = (C.c_int64 * ns)(*[int(v) for v in n_per_sys])
    h = C.c_void_p()
    rc = lib().md_create_batch(ns, S, P, N, C.byref(h))
    _check(None, rc)
    return h


def md_set_stream(h, stream) -> None:
    ptr = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
    _check(h, lib().md_set_stream(h, C.c_void_p(ptr) if ptr else None))


def md_set_state(h, x, v=None, type=None, mol=None, constrained=None, step0: int = 0) -> None:
    x_, xp = _host(x, np.float64, (-1, 3))
    v_, vp = _host(v, np.float64, (-1, 3))
    t_, tp = _host(type, np.int32)
    m_, mp = _host(mol, np.int32)
    c_, cp = _host(constrained, np.uint8)
    _check(h, lib().md_set_state(h, xp, vp, tp, mp, cp, int(step0)))


def md_set_state_device(h, d_x, d_v=None, d_type=None, d_mol=None, d_con=None, step0: int = 0) -> None:
    _check(h, lib().md_set_state_device(h, _dptr(d_x), _dptr(d_v), _dptr(d_type), _dptr(d_mol),
                                        _dptr(d_con), int(step0)))


def md_restore(h, x, p_half, step: int) -> None:
    x_, xp = _host(x, np.float64, (-1, 3))
    p_, pp = _host(p_half, np.float64, (-1, 3))
    _check(h, lib().md_restore(h, xp, pp, int(step)))


def md_step(h, nsteps: int) -> None:
    _check(h, lib().md_step(h, int(nsteps)))


def md_sync(h) -> None:
    _check(h, lib().md_sync(h))


def md_status(h) -> int:
    f = C.c_uint32()
    _check(h, lib().md_status(h, C.byref(f)))
    return f.value


def md_info(h):
    n, ns, st = C.c_int64(), C.c_int32(), C.c_uint64()
    _check(h, lib().md_info(h, C.byref(n), C.byref(ns), C.byref(st)))
    return {"n": n.value, "nsys": ns.value, "step": st.value}


def md_get_state(h, want=("x", "v", "p_half")):
    n = md_info(h)["n"]
    out = {k: np.zeros((n, 3)) for k in want}
    ptr = {k: (out[k].ctypes.data_as(C.c_void_p) if k in out else None) for k in ("x", "v", "p_half")}
    st = C.c_uint64()
    _check(h, lib().md_get_state(h, ptr["x"], ptr["v"], ptr["p_half"], C.byref(st)))
    out["step"] = st.value
    return out


def md_get_state_device(h, d_x=None, d_v=None, d_p_half=None) -> None:
    _check(h, lib().md_get_state_device(h, _dptr(d_x), _dptr(d_v), _dptr(d_p_half)))


def md_forces(h):
    n = md_info(h)["n"]
    f, u = np.zeros((n, 3)), np.zeros(n)
    _check(h, lib().md_forces(h, f.ctypes.data_as(C.c_void_p), u.ctypes.data_as(C.c_void_p)))
    return f, u


def md_constraint_residual(h):
    a, b, c = C.c_double(), C.c_double(), C.c_double()
    _check(h, lib().md_constraint_residual(h, C.byref(a), C.byref(b), C.byref(c)))
    return {"max_g_over_gradg": a.value, "max_abs_g": b.value, "max_n_dot_v": c.value}


def md_observables(h):
    ns = md_info(h)["nsys"]
    arr = (md_obs * ns)()
    nw = C.c_int32()
    _check(h, lib().md_observables(h, arr, ns, C.byref(nw)))
    return [{f: getattr(arr[i], f) for f, _ in md_obs._fields_} for i in range(nw.value)]


def md_last_launch_count(h) -> int:
    v = C.c_int64()
    _check(h, lib().md_last_launch_count(h, C.byref(v)))
    return v.value


def md_grid_info(h, sys: int = 0):
    lo, cs = (C.c_double * 3)(), (C.c_double * 3)()
    nc = (C.c_int32 * 3)()
    base, hashed = C.c_uint32(), C.c_int32()
    _check(h, lib().md_grid_info(h, int(sys), lo, cs, nc, C.byref(base), C.byref(hashed)))
    return {"lo": np.array(lo[:]), "cs": np.array(cs[:]), "nc": np.array(nc[:]), "base": base.value,
            "hashed": hashed.value}


def md_measure_fma_peak(precision: str = "fp64", trials: int = 5) -> float:
    """Measured FMA instructions per second of the current device
    (float64 for "fp64", float32 for "mixed")."""
    out = C.c_double()
    rc = lib().md_measure_fma_peak(PRECISION[precision] if isinstance(precision, str) else int(precision),
                                   int(trials), C.byref(out))
    if rc:
        raise MdError(rc, md_last_error(None))
    return out.value


def md_cell_list(h):
    n = md_info(h)["n"]
    nb = C.c_uint32()
    _check(h, lib().md_cell_list(h, None, None, None, C.byref(nb)))
    ids, cells = np.zeros(n, np.uint32), np.zeros(n, np.uint32)
    start = np.zeros(nb.value + 1, np.uint32)
    _check(h, lib().md_cell_list(h, ids.ctypes.data_as(C.c_void_p), cells.ctypes.data_as(C.c_void_p),
                                 start.ctypes.data_as(C.c_void_p), C.byref(nb)))
    return {"sorted_ids": ids, "sorted_cells": cells, "bucket_start": start}


def md_profile_step(h, nsteps: int = 1):
    """Mean duration (ms) of each kernel of a step, keyed by kernel name."""
    buf = (C.c_double * 16)()
    nk = C.c_int32()
    _check(h, lib().md_profile_step(h, int(nsteps), buf, 16, C.byref(nk)))
    return {lib().md_profile_kernel_name(h, i).decode(): buf[i] for i in range(nk.value)}


def md_forces_noalloc(surface: dict | None, params: dict, n: int, d_x, d_f, d_type=None, d_mol=None,
                      d_con=None, d_u=None, stream=None) -> None:
    """Forces of one system at device positions d_x into device d_f (and d_u)
    without any device allocation (the library's fixed scratch array is used;
    at most 65,536 particles). Device arguments are ints or objects with
    data_ptr(); stream is a cudaStream_t or an object with cuda_stream."""
    S, P = make_surface(surface), make_params(params)
    sptr = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
    rc = lib().md_forces_noalloc(C.byref(S), C.byref(P), int(n), _dptr(d_x), _dptr(d_type), _dptr(d_mol),
                                 _dptr(d_con), _dptr(d_f), _dptr(d_u), C.c_void_p(sptr) if sptr else None)
    _check(None, rc)


def md_check_conversions(values) -> tuple[np.ndarray, np.ndarray]:
    """float64 values rounded to float32 and widened back, by the device's
    integer-pipe conversions (a diagnostic of the mixed path)."""
    v = np.ascontiguousarray(values, dtype=np.float64)
    f = np.empty(v.shape, np.float32)
    d = np.empty(v.shape, np.float64)
    _check(None, lib().md_check_conversions(v.ctypes.data, v.size, f.ctypes.data, d.ctypes.data))
    return f, d


def md_set_option(h, key: int, value: int) -> None:
    _check(h, lib().md_set_option(h, int(key), int(value)))


def md_set_neighbor_list(h, skin: float, max_neighbors: int = 64) -> None:
    """Verlet neighbour list with the given skin (<= 0: off); the handle's
    cell edge must be at least the largest cutoff + skin."""
    _check(h, lib().md_set_neighbor_list(h, float(skin), int(max_neighbors)))


def md_get_option(h, key: int) -> int:
    v = C.c_int64()
    _check(h, lib().md_get_option(h, int(key), C.byref(v)))
    return v.value


def md_last_error(h=None) -> str:
    r = lib().md_last_error(h)
    return r.decode() if r else ""


def md_destroy(h) -> None:
    if h:
        lib().md_destroy(h)


# ---------------------------------------------------------------------------
# convenience: a batch of systems described by the dictionaries of `inputs`
# ---------------------------------------------------------------------------
class Simulation:
    """Owns one handle for a list of system dicts (surface, params, n, x, v,
    type, constrained), all advanced together."""

    def __init__(self, systems: list[dict], stream=None):
        self.systems = systems
        self.n = int(sum(s["n"] for s in systems))
        if len(systems) == 1:
            s = systems[0]
            self.h = md_create(s["surface"], s["params"], s["n"])
        else:
            self.h = md_create_batch([s["surface"] for s in systems], [s["params"] for s in systems],
                                     [s["n"] for s in systems])
        if stream is not None:
            md_set_stream(self.h, stream)

    def set_state(self, step0: int = 0):
        cat = lambda k: np.concatenate([s[k] for s in self.systems]) if self.n else None  # noqa: E731
        mol = None
        if any("mol" in s for s in self.systems):
            mol = np.concatenate([s.get("mol") for s in self.systems])
        md_set_state(self.h, cat("x"), cat("v"), cat("type"), mol, cat("constrained"), step0)

    def step(self, n: int = 1):
        md_step(self.h, n)

    def sync(self):
        md_sync(self.h)

    def state(self):
        return md_get_state(self.h)

    def forces(self):
        return md_forces(self.h)

    def residual(self):
        return md_constraint_residual(self.h)

    def observables(self):
        return md_observables(self.h)

    def close(self):
        if getattr(self, "h", None):
            md_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
