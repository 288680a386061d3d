"""Oracle: a plain, slow float64 CPU reference of the constrained Langevin
time step of Paquay & Kusters (Algorithm 1, Algorithm S1, Eq. S1).

TEST INFRASTRUCTURE. Only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package. The product (the
CUDA library and its binding) never imports, links or runs it, and this
package imports nothing from the product. The C source ``oracle.c`` holds all
of the arithmetic; this module only marshals numpy arrays through ctypes.

Parity status: every exported routine is pinned by the ``-m "not gpu"``
tests (Philox known-answer vectors, closed-form Newton roots, brute force,
finite differences, the Langevin stationary variances derived from
Algorithm S1, the plane and sphere diffusion laws of SI Section S1.3,
energy conservation) except the diffusion coefficient of interacting
particles, for which the paper fixes no value (parity unpinned).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

MAXT = 8
SURF_KINDS = {"none": 0, "plane": 1, "sphere": 2, "ellipsoid": 3, "torus": 4,
              "gaussian_bump": 5, "cylinder": 6, "xy2d": 7, "thylakoid": 8}


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, -O2, no FMA contraction so
    that x86 and Arm give the same bits)."""
    if force or not os.path.exists(_LIB_PATH) or \
            os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-ffp-contract=off",
               "-fno-fast-math", "-Wall", "-o", tmp, _SRC, "-lm"]
        # OpenMP over the independent per-particle loops where the compiler has it
        if subprocess.run(cmd[:1] + ["-fopenmp"] + cmd[1:], capture_output=True).returncode != 0:
            subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Surface(C.Structure):
    _fields_ = [("kind", C.c_int32), ("pad", C.c_int32),
                ("c", C.c_double * 3), ("p", C.c_double * 4)]


class Params(C.Structure):
    _fields_ = [("dt", C.c_double), ("kT", C.c_double), ("gamma", C.c_double),
                ("tol", C.c_double),
                ("max_newton", C.c_int32), ("ntypes", C.c_int32),
                ("beads_per_mol", C.c_int32), ("exclude_intramol", C.c_int32),
                ("mass", C.c_double * MAXT),
                ("eps", (C.c_double * MAXT) * MAXT),
                ("sigma", (C.c_double * MAXT) * MAXT),
                ("rcut", (C.c_double * MAXT) * MAXT),
                ("box_lo", C.c_double * 3), ("box_hi", C.c_double * 3),
                ("periodic", C.c_int32 * 3), ("wall_enable", C.c_int32),
                ("bond_k", C.c_double), ("bond_r0", C.c_double),
                ("wall_lo_z", C.c_double), ("wall_hi_z", C.c_double),
                ("wall_eps", C.c_double), ("wall_sigma", C.c_double),
                ("seed", C.c_uint64), ("replica", C.c_uint32),
                ("force_mode", C.c_int32), ("pair_form", C.c_int32),
                ("angle_k", C.c_double), ("angle_theta0", C.c_double),
                ("bond_r0_mix", C.c_int32), ("wall_kind", C.c_int32),
                ("wall_radius", C.c_double), ("wall_center", C.c_double * 3)]


_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_up = np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")
_u32p = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB_PATH)
            L.orc_philox4x32_10.argtypes = [_u32p, _u32p, _u32p]
            L.orc_gauss3.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint64, _dp]
            L.orc_surface_g.restype = C.c_double
            L.orc_surface_g.argtypes = [C.POINTER(Surface), C.POINTER(Params), _dp, _dp]
            L.orc_position_half.restype = C.c_int
            L.orc_position_half.argtypes = [C.POINTER(Surface), C.POINTER(Params), _dp, _dp, _dp,
                                            C.c_double, _dp, _dp, C.POINTER(C.c_double),
                                            C.POINTER(C.c_int32)]
            L.orc_momentum_half.restype = C.c_int
            L.orc_momentum_half.argtypes = [C.POINTER(Surface), C.POINTER(Params), _dp, _dp, _dp,
                                            C.c_double, _dp, C.POINTER(C.c_double),
                                            C.POINTER(C.c_int32)]
            L.orc_pair_forces_brute.argtypes = [C.POINTER(Params), C.c_int64, _dp, _ip, _ip, _dp, _dp]
            L.orc_pair_forces_cells.restype = C.c_int
            L.orc_pair_forces_cells.argtypes = [C.POINTER(Params), C.c_int64, _dp, _ip, _ip, _dp, _dp]
            L.orc_bond_wall_forces.restype = C.c_int
            L.orc_bond_wall_forces.argtypes = [C.POINTER(Params), C.c_int64, _dp, C.c_void_p, C.c_void_p, _dp,
                                               _dp]
            L.orc_create.restype = C.c_void_p
            L.orc_create.argtypes = [C.POINTER(Surface), C.POINTER(Params), C.c_int64]
            L.orc_destroy.argtypes = [C.c_void_p]
            L.orc_set_state.restype = C.c_int
            L.orc_set_state.argtypes = [C.c_void_p, _dp, C.c_void_p, C.c_void_p, C.c_void_p,
                                        C.c_void_p, C.c_uint64]
            L.orc_step.restype = C.c_int64
            L.orc_step.argtypes = [C.c_void_p, C.c_int64]
            L.orc_get_state.argtypes = [C.c_void_p, _dp, _dp, _dp, _dp, C.POINTER(C.c_uint64)]
            L.orc_get_forces.argtypes = [C.c_void_p, _dp, _dp]
            L.orc_residual.argtypes = [C.c_void_p, _dp]
            L.orc_observables.argtypes = [C.c_void_p, _dp]
            L.orc_newton_stats.argtypes = [C.c_void_p, _i64p]
            L.orc_wall_violation.restype = C.c_int32
            L.orc_wall_violation.argtypes = [C.c_void_p]
            L.orc_sys_forces.restype = C.c_int
            L.orc_sys_forces.argtypes = [C.c_void_p]
            L.orc_force_on.argtypes = [C.POINTER(Params), C.c_int64, _dp, _ip, _ip, C.c_void_p,
                                       C.c_int64, _dp, C.POINTER(C.c_double)]
            L.orc_force_scale.argtypes = [C.POINTER(Params), C.c_int64, _dp, _ip, _ip, C.c_void_p, _dp]
            L.orc_particle_advance.restype = C.c_int
            L.orc_particle_advance.argtypes = [C.POINTER(Surface), C.POINTER(Params), C.c_int64, _dp,
                                               _ip, _ip, C.c_void_p, C.c_int64, _dp, C.c_uint64,
                                               C.c_int, _dp, _dp, _dp]
            L.orc_set_threads.argtypes = [C.c_int]
            L.orc_set_threads.restype = C.c_int
            L.orc_set_threads(1)  # one thread unless set_threads asks for more
            _lib = L
    return _lib


def set_threads(k: int) -> int:
    """Threads of the oracle's per-particle loops (OpenMP; 1 if it was built
    without). Results are the same at any count. Returns the count in use."""
    return int(lib().orc_set_threads(int(k)))


# ---------------------------------------------------------------------------
# dict -> struct (field names follow the library's md_params; the conversion
# is written here independently of the product binding)
# ---------------------------------------------------------------------------
def make_surface(surf: dict | None) -> Surface:
    s = Surface()
    surf = surf or {"kind": "none"}
    kind = surf.get("kind", "none")
    s.kind = SURF_KINDS[kind] if isinstance(kind, str) else int(kind)
    for k, v in enumerate(surf.get("center", (0.0, 0.0, 0.0))):
        s.c[k] = float(v)
    for k, v in enumerate(surf.get("p", ())):
        s.p[k] = float(v)
    return s


def make_params(prm: dict, force_mode: int = 0) -> Params:
    P = Params()
    P.dt = prm["dt"]
    P.kT = prm.get("kT", 1.0)
    P.gamma = prm.get("gamma", 1.0)
    P.tol = prm.get("rattle_tol", 1e-12)
    P.max_newton = prm.get("max_newton", 30)
    nt = prm.get("ntypes", 1)
    P.ntypes = nt
    mass = prm.get("mass", [1.0] * nt)
    for a in range(MAXT):
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
    P.force_mode = force_mode
    P.pair_form = int(prm.get("pair_form", 0))
    P.angle_k = float(prm.get("angle_k", 0.0))
    P.angle_theta0 = float(prm.get("angle_theta0", 0.0))
    P.bond_r0_mix = int(prm.get("bond_r0_mix", 0))
    P.wall_kind = int(prm.get("wall_kind", 0))
    P.wall_radius = float(prm.get("wall_radius", 0.0))
    for k in range(3):
        P.wall_center[k] = float(prm.get("wall_center", (0.0, 0.0, 0.0))[k])
    return P


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a if shape is None else a.reshape(shape)


# ---------------------------------------------------------------------------
# Low-level routines
# ---------------------------------------------------------------------------
def philox4x32_10(ctr, key) -> np.ndarray:
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(np.ascontiguousarray(ctr, dtype=np.uint32),
                            np.ascontiguousarray(key, dtype=np.uint32), out)
    return out


def gauss3(seed: int, replica: int, pid: int, step: int) -> np.ndarray:
    out = np.zeros(3)
    lib().orc_gauss3(seed, replica, pid, step, out)
    return out


def surface_g(surf: dict, prm: dict, x) -> tuple[float, np.ndarray]:
    n = np.zeros(3)
    S, P = make_surface(surf), make_params(prm)
    g = lib().orc_surface_g(C.byref(S), C.byref(P), _f64(x), n)
    return g, n


def position_half(surf, prm, x, p, f, m=1.0):
    """Algorithm 1, position half for one particle: (x_new, p_half, lambda,
    iterations, status)."""
    S, P = make_surface(surf), make_params(prm)
    xn, ph = np.zeros(3), np.zeros(3)
    lam, its = C.c_double(), C.c_int32()
    st = lib().orc_position_half(C.byref(S), C.byref(P), _f64(x), _f64(p), _f64(f), m,
                                 xn, ph, C.byref(lam), C.byref(its))
    return xn, ph, lam.value, its.value, st


def momentum_half(surf, prm, x_new, p_half, f_new, m=1.0):
    """Algorithm 1, momentum half for one particle: (p_new, mu, iterations, status)."""
    S, P = make_surface(surf), make_params(prm)
    pn = np.zeros(3)
    mu, its = C.c_double(), C.c_int32()
    st = lib().orc_momentum_half(C.byref(S), C.byref(P), _f64(x_new), _f64(p_half),
                                 _f64(f_new), m, pn, C.byref(mu), C.byref(its))
    return pn, mu.value, its.value, st


def pair_forces(prm, x, type_=None, mol=None, mode="brute"):
    """Truncated-shifted LJ forces (Eq. S1): (f [n,3], u [n])."""
    x = _f64(x, (-1, 3))
    n = x.shape[0]
    t = np.zeros(n, np.int32) if type_ is None else np.ascontiguousarray(type_, np.int32)
    mo = np.arange(n, dtype=np.int32) if mol is None else np.ascontiguousarray(mol, np.int32)
    f, u = np.zeros((n, 3)), np.zeros(n)
    P = make_params(prm)
    if mode == "brute":
        lib().orc_pair_forces_brute(C.byref(P), n, x, t, mo, f, u)
    else:
        if lib().orc_pair_forces_cells(C.byref(P), n, x, t, mo, f, u):
            raise MemoryError("oracle cell list allocation failed")
    return f, u


def bond_wall_forces(prm, x, constrained=None, type_=None):
    """Bonded (bonds, bend angles) and wall forces and per-particle energies
    (SI S3.2); returns (f, u, behind_a_wall)."""
    x = _f64(x, (-1, 3))
    n = x.shape[0]
    f, u = np.zeros((n, 3)), np.zeros(n)
    con = None if constrained is None else np.ascontiguousarray(constrained, np.uint8)
    t = None if type_ is None else np.ascontiguousarray(type_, np.int32)
    P = make_params(prm)
    bad = lib().orc_bond_wall_forces(C.byref(P), n, x, None if t is None else t.ctypes.data,
                                     None if con is None else con.ctypes.data, f, u)
    return f, u, bad


def _arrays(x, type_, mol, constrained, surf, prm):
    x = _f64(x, (-1, 3))
    n = x.shape[0]
    t = np.zeros(n, np.int32) if type_ is None else np.ascontiguousarray(type_, np.int32)
    if mol is None:
        bpm = prm.get("beads_per_mol", 0)
        mo = (np.arange(n) // bpm if bpm > 1 else np.arange(n)).astype(np.int32)
    else:
        mo = np.ascontiguousarray(mol, np.int32)
    if constrained is None:
        kind = (surf or {}).get("kind", "none")
        con = np.full(n, 0 if kind in ("none", "xy2d") else 1, np.uint8)
    else:
        con = np.ascontiguousarray(constrained, np.uint8)
    return x, t, mo, con


def force_on(prm, x, i, type_=None, mol=None, constrained=None, surf=None):
    """Force and energy on particle i only (all pairs with i, its bonds and walls)."""
    x, t, mo, con = _arrays(x, type_, mol, constrained, surf, prm)
    f = np.zeros(3)
    u = C.c_double()
    P = make_params(prm)
    lib().orc_force_on(C.byref(P), x.shape[0], x, t, mo, con.ctypes.data, int(i), f, C.byref(u))
    return f, u.value


def force_scale(prm, x, type_=None, mol=None, constrained=None, surf=None):
    """Per particle, the sum of the force magnitudes of its pair, bond and wall terms."""
    x, t, mo, con = _arrays(x, type_, mol, constrained, surf, prm)
    out = np.zeros(x.shape[0])
    P = make_params(prm)
    lib().orc_force_scale(C.byref(P), x.shape[0], x, t, mo, con.ctypes.data, out)
    return out


def particle_advance(surf, prm, x, i, p_in, step, first, type_=None, mol=None, constrained=None):
    """Algorithm S1 for particle i: (p^k, x^{k+1}, p^{k+1/2}, status)."""
    x, t, mo, con = _arrays(x, type_, mol, constrained, surf, prm)
    S, P = make_surface(surf), make_params(prm)
    pk, xn, phn = np.zeros(3), np.zeros(3), np.zeros(3)
    st = lib().orc_particle_advance(C.byref(S), C.byref(P), x.shape[0], x, t, mo, con.ctypes.data,
                                    int(i), _f64(p_in), int(step), int(first), pk, xn, phn)
    return pk, xn, phn, st


# ---------------------------------------------------------------------------
# A system advanced by Algorithm S1
# ---------------------------------------------------------------------------
class System:
    """One system of n particles on one surface, stepped by Algorithm S1."""

    def __init__(self, surf: dict | None, prm: dict, n: int, force_mode: str = "auto"):
        mode = {"auto": 0, "brute": 1, "cells": 2}[force_mode]
        self.S, self.P, self.n = make_surface(surf), make_params(prm, mode), int(n)
        self._h = lib().orc_create(C.byref(self.S), C.byref(self.P), self.n)
        if not self._h:
            raise MemoryError("orc_create failed")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_destroy(h)
            self._h = None

    def set_state(self, x, v=None, type_=None, mol=None, constrained=None, step0=0):
        n = self.n
        x = _f64(x, (n, 3))
        keep = []

        def ptr(a, dt):
            if a is None:
                return None
            a = np.ascontiguousarray(a, dtype=dt)
            keep.append(a)
            return a.ctypes.data
        st = lib().orc_set_state(self._h, x, ptr(v, np.float64), ptr(type_, np.int32),
                                 ptr(mol, np.int32), ptr(constrained, np.uint8), step0)
        if st == 1:
            raise ValueError("a constrained particle is off its surface")
        if st != 0:
            raise RuntimeError(f"orc_set_state failed ({st})")

    def step(self, nsteps: int = 1) -> int:
        r = lib().orc_step(self._h, nsteps)
        if r < 0:
            raise RuntimeError("oracle step failed")
        return r

    def state(self):
        n = self.n
        x, v, ph, F = np.zeros((n, 3)), np.zeros((n, 3)), np.zeros((n, 3)), np.zeros((n, 3))
        st = C.c_uint64()
        lib().orc_get_state(self._h, x, v, ph, F, C.byref(st))
        return {"x": x, "v": v, "p_half": ph, "F": F, "step": st.value}

    def forces(self):
        f, u = np.zeros((self.n, 3)), np.zeros(self.n)
        lib().orc_get_forces(self._h, f, u)
        return f, u

    def recompute_forces(self):
        if lib().orc_sys_forces(self._h):
            raise MemoryError("oracle force allocation failed")
        return self.forces()

    def residual(self):
        out = np.zeros(3)
        lib().orc_residual(self._h, out)
        return {"max_g_over_gradg": out[0], "max_abs_g": out[1], "max_n_dot_v": out[2]}

    def observables(self):
        out = np.zeros(6)
        lib().orc_observables(self._h, out)
        return {"kinetic": out[0], "potential": out[1], "kT": out[2], "msd": out[3],
                "r0_dot_rt": out[4], "ndof": int(out[5])}

    def newton_stats(self):
        out = np.zeros(3, dtype=np.int64)
        lib().orc_newton_stats(self._h, out)
        return {"fail": int(out[0]), "floor": int(out[1]), "iters": int(out[2])}

    def wall_violation(self) -> bool:
        return bool(lib().orc_wall_violation(self._h))
