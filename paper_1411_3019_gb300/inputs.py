"""Seeded synthetic inputs shaped like the paper's workloads.

This module serves both the CUDA path and the oracle and therefore holds
none of the method's arithmetic: no Newton solve, no force, no noise, no
projection. It only draws positions uniformly (by area) on a surface or in a
volume with overlaps rejected (random sequential addition), Maxwell
velocities, and the parameter dictionaries of the workloads. Surfaces are
sampled from their parametrisations, never from g(x).

Every generator takes a seed and uses numpy's counter-based Philox bit
generator, so a given seed gives the same arrays on every machine.

Area fraction (Section 3.2): phi = N A_p / A with A_p = pi d0^2 / 4 and
d0 = 2^{1/6} sigma, the WCA cutoff.
"""
from __future__ import annotations

import math

import numpy as np

D0 = 2.0 ** (1.0 / 6.0)
A_P = math.pi * D0 * D0 / 4.0
WCA_RC = D0


def rng(seed: int, stream: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=[seed & 0xFFFFFFFFFFFFFFFF, stream]))


# ---------------------------------------------------------------------------
# parameters
# ---------------------------------------------------------------------------
def wca_params(ntypes: int = 1, **over) -> dict:
    """WCA particles (eps = sigma = m = 1, cutoff 2^{1/6} sigma), kT = gamma = 1."""
    eps = np.zeros((ntypes, ntypes))
    sig = np.zeros((ntypes, ntypes))
    rc = np.zeros((ntypes, ntypes))
    eps[:, :] = 1.0
    sig[:, :] = 1.0
    rc[:, :] = WCA_RC
    prm = dict(dt=0.002, kT=1.0, gamma=1.0, rattle_tol=1e-10, max_newton=30,
               frozen_normal=0, precision="mixed", ntypes=ntypes, mass=[1.0] * ntypes,
               eps=eps, sigma=sig, rcut=rc, box_lo=(0.0, 0.0, 0.0), box_hi=(0.0, 0.0, 0.0),
               periodic=(0, 0, 0), beads_per_mol=0, bond_k=0.0, bond_r0=0.0,
               exclude_intramol=0, wall_enable=0, wall_lo_z=0.0, wall_hi_z=0.0,
               wall_eps=1.0, wall_sigma=1.0, seed=1, replica=0, cell_size=0.0)
    prm.update(over)
    return prm


def noninteracting(prm: dict) -> dict:
    """The same parameters with every pair term switched off."""
    out = dict(prm)
    nt = prm["ntypes"]
    out["eps"] = np.zeros((nt, nt))
    out["rcut"] = np.zeros((nt, nt))
    return out


# ---------------------------------------------------------------------------
# surface areas (for the area fraction only)
# ---------------------------------------------------------------------------
def ellipsoid_area(a: float, b: float, c: float, n: int = 2000) -> float:
    """Area of the ellipsoid by midpoint quadrature over the sphere angles."""
    th = (np.arange(n) + 0.5) * math.pi / n
    ph = (np.arange(2 * n) + 0.5) * math.pi / n
    T, P = np.meshgrid(th, ph, indexing="ij")
    st, ct, sp, cp = np.sin(T), np.cos(T), np.sin(P), np.cos(P)
    nx, ny, nz = b * c * st * st * cp, a * c * st * st * sp, a * b * st * ct
    dA = np.sqrt(nx * nx + ny * ny + nz * nz)
    return float(dA.sum() * (math.pi / n) * (math.pi / n))


def torus_area(R: float, r: float) -> float:
    return 4.0 * math.pi ** 2 * R * r


def bump_area(L: float, A: float, w: float, n: int = 1500) -> float:
    h = L / n
    u = (np.arange(n) + 0.5) * h - L / 2
    X, Y = np.meshgrid(u, u, indexing="ij")
    e = A * np.exp(-(X * X + Y * Y) / (2 * w * w))
    gx, gy = -e * X / (w * w), -e * Y / (w * w)
    return float(np.sqrt(1 + gx * gx + gy * gy).sum() * h * h)


# ---------------------------------------------------------------------------
# uniform-by-area samplers (parametrisations + rejection on the area element)
# ---------------------------------------------------------------------------
def sample_surface(surf: dict, n: int, g: np.random.Generator, box=None) -> np.ndarray:
    kind = surf["kind"]
    c = np.asarray(surf.get("center", (0.0, 0.0, 0.0)), dtype=np.float64)
    p = surf.get("p", ())
    if kind == "sphere":
        v = g.standard_normal((n, 3))
        v /= np.linalg.norm(v, axis=1, keepdims=True)
        return c + p[0] * v
    if kind == "ellipsoid":
        a, b, cc = p[0], p[1], p[2]
        out = np.empty((0, 3))
        mx = max(b * cc, a * cc, a * b)
        while out.shape[0] < n:
            m = 2 * (n - out.shape[0]) + 64
            v = g.standard_normal((m, 3))
            v /= np.linalg.norm(v, axis=1, keepdims=True)
            w = np.sqrt((b * cc * v[:, 0]) ** 2 + (a * cc * v[:, 1]) ** 2 + (a * b * v[:, 2]) ** 2)
            keep = g.random(m) < w / mx
            out = np.vstack([out, v[keep] * np.array([a, b, cc])])
        return c + out[:n]
    if kind == "torus":
        R, r = p[0], p[1]
        out = np.empty((0, 3))
        while out.shape[0] < n:
            m = 2 * (n - out.shape[0]) + 64
            th = g.random(m) * 2 * math.pi
            keep = g.random(m) < (R + r * np.cos(th)) / (R + r)
            th = th[keep]
            ph = g.random(th.shape[0]) * 2 * math.pi
            rr = R + r * np.cos(th)
            out = np.vstack([out, np.stack([rr * np.cos(ph), rr * np.sin(ph), r * np.sin(th)], 1)])
        return c + out[:n]
    if kind == "gaussian_bump":
        A, w = p[0], p[1]
        lo, hi = np.asarray(box[0], float), np.asarray(box[1], float)
        L = hi - lo
        out = np.empty((0, 3))
        while out.shape[0] < n:
            m = 2 * (n - out.shape[0]) + 64
            xy = lo[:2] + g.random((m, 2)) * L[:2]
            d = xy - c[:2]
            d -= L[:2] * np.floor(d / L[:2] + 0.5)
            e = A * np.exp(-(d ** 2).sum(1) / (2 * w * w))
            slope2 = (e / (w * w)) ** 2 * (d ** 2).sum(1)
            mx = 1.0 + (A / (w * math.sqrt(math.e))) ** 2
            keep = g.random(m) < np.sqrt(1 + slope2) / math.sqrt(mx)
            z = c[2] + e[keep]
            out = np.vstack([out, np.column_stack([xy[keep], z])])
        return out[:n]
    if kind == "xy2d":
        lo, hi = np.asarray(box[0], float), np.asarray(box[1], float)
        xy = lo[:2] + g.random((n, 2)) * (hi - lo)[:2]
        return np.column_stack([xy, np.full(n, c[2])])
    if kind == "plane":
        lo, hi = np.asarray(box[0], float), np.asarray(box[1], float)
        nrm = np.asarray(p[:3], float)
        if not (nrm[0] == 0 and nrm[1] == 0):
            raise ValueError("the plane sampler covers planes normal to z")
        xy = lo[:2] + g.random((n, 2)) * (hi - lo)[:2]
        return np.column_stack([xy, np.full(n, c[2])])
    if kind == "cylinder":
        R, ax = p[0], int(p[1])
        lo, hi = np.asarray(box[0], float), np.asarray(box[1], float)
        t = lo[ax] + g.random(n) * (hi - lo)[ax]
        ph = g.random(n) * 2 * math.pi
        other = [k for k in range(3) if k != ax]
        out = np.empty((n, 3))
        out[:, ax] = t
        out[:, other[0]] = c[other[0]] + R * np.cos(ph)
        out[:, other[1]] = c[other[1]] + R * np.sin(ph)
        return out
    raise ValueError(f"no sampler for surface {kind!r}")


# ---------------------------------------------------------------------------
# random sequential addition with a hashed grid (groups never conflict)
# ---------------------------------------------------------------------------
def _keys(cells: np.ndarray, group: np.ndarray) -> np.ndarray:
    c = cells.astype(np.int64) + 32768
    return (group.astype(np.int64) << 48) | (c[:, 0] << 32) | (c[:, 1] << 16) | c[:, 2]


def _conflicts(cand, cgrp, ref, rgrp, dmin, periodic, L, lo, exclude_self=False):
    """For each candidate: does it lie closer than dmin to a reference point
    of the same group? (exclude_self: cand and ref are the same array and a
    point conflicts only with an earlier index.)"""
    n = cand.shape[0]
    bad = np.zeros(n, bool)
    if ref.shape[0] == 0 or n == 0:
        return bad
    cs = dmin
    ncell = np.where(periodic, np.maximum(np.floor(L / cs), 1), 1 << 14).astype(np.int64)

    def cell_of(pts):
        rel = pts - lo
        c = np.floor(rel / cs).astype(np.int64)
        for k in range(3):
            if periodic[k]:
                c[:, k] = np.mod(np.floor(rel[:, k] / (L[k] / ncell[k])).astype(np.int64), ncell[k])
        return c

    rc, cc = cell_of(ref), cell_of(cand)
    rk = _keys(rc, rgrp)
    order = np.argsort(rk, kind="stable")
    rk_s, ref_s, ridx_s = rk[order], ref[order], order
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                nc = cc + np.array([dx, dy, dz])
                for k in range(3):
                    if periodic[k]:
                        nc[:, k] = np.mod(nc[:, k], ncell[k])
                nk = _keys(nc, cgrp)
                a = np.searchsorted(rk_s, nk, "left")
                b = np.searchsorted(rk_s, nk, "right")
                occ = int((b - a).max()) if n else 0
                for t in range(occ):
                    idx = a + t
                    ok = idx < b
                    if not ok.any():
                        continue
                    j = np.where(ok, idx, 0)
                    d = cand - ref_s[j]
                    for k in range(3):
                        if periodic[k]:
                            d[:, k] -= L[k] * np.floor(d[:, k] / L[k] + 0.5)
                    close = ok & ((d * d).sum(1) < dmin * dmin)
                    if exclude_self:
                        close &= ridx_s[j] < np.arange(n)
                    bad |= close
    return bad


def rsa(sampler, counts, dmin, g, periodic=(0, 0, 0), box=None, fixed=None, fixed_group=None,
        max_rounds=400, sampler_multi=None):
    """Random sequential addition: group k receives counts[k] points from
    sampler(k, m) (or sampler_multi(group_ids) for all groups at once) with no
    two points of one group (nor a point and a fixed point of that group)
    closer than dmin."""
    counts = np.asarray(counts, dtype=np.int64)
    periodic = np.asarray(periodic, bool)
    if box is None:
        lo, L = np.zeros(3), np.ones(3)
    else:
        lo = np.asarray(box[0], float)
        L = np.asarray(box[1], float) - lo
    have = np.zeros(counts.shape[0], np.int64)
    acc_pts, acc_grp = [], []
    pts = np.empty((0, 3)) if fixed is None else np.asarray(fixed, float)
    grp = np.empty(0, np.int64) if fixed is None else np.asarray(fixed_group, np.int64)
    for _ in range(max_rounds):
        need = counts - have
        if (need <= 0).all():
            break
        ks = np.nonzero(need > 0)[0]
        m = (need[ks] * 1.3).astype(np.int64) + 16
        cg = np.repeat(ks, m)
        if sampler_multi is not None:
            cand = sampler_multi(cg)
        else:
            cand = np.vstack([sampler(int(k), int(mk)) for k, mk in zip(ks, m)])
        active = need[grp] > 0  # points of finished groups can no longer conflict
        bad = _conflicts(cand, cg, pts[active], grp[active], dmin, periodic, L, lo)
        cand, cg = cand[~bad], cg[~bad]
        bad = _conflicts(cand, cg, cand, cg, dmin, periodic, L, lo, exclude_self=True)
        cand, cg = cand[~bad], cg[~bad]
        order = np.argsort(cg, kind="stable")
        cand, cg = cand[order], cg[order]
        first = np.searchsorted(cg, cg, "left")
        rank = np.arange(cg.shape[0]) - first
        keep = rank < need[cg]
        cand, cg = cand[keep], cg[keep]
        have += np.bincount(cg, minlength=counts.shape[0])
        acc_pts.append(cand)
        acc_grp.append(cg)
        pts = np.vstack([pts, cand])
        grp = np.concatenate([grp, cg])
    if (have < counts).any():
        k = int(np.nonzero(have < counts)[0][0])
        raise RuntimeError(f"RSA could not place {counts[k]} points in group {k}")
    allp = np.vstack(acc_pts) if acc_pts else np.empty((0, 3))
    allg = np.concatenate(acc_grp) if acc_grp else np.empty(0, np.int64)
    order = np.argsort(allg, kind="stable")
    allp, allg = allp[order], allg[order]
    bounds = np.concatenate([[0], np.cumsum(counts)])
    return [allp[bounds[k]:bounds[k + 1]] for k in range(counts.shape[0])]


def maxwell(n: int, kT: float, mass, g: np.random.Generator) -> np.ndarray:
    m = np.broadcast_to(np.asarray(mass, float), (n,))
    return g.standard_normal((n, 3)) * np.sqrt(kT / m)[:, None]


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------
def _system(name, surface, params, x, v, type_=None, constrained=None):
    n = x.shape[0]
    return dict(name=name, surface=surface, params=params, n=n,
                x=np.ascontiguousarray(x, np.float64), v=np.ascontiguousarray(v, np.float64),
                type=np.zeros(n, np.int32) if type_ is None else np.ascontiguousarray(type_, np.int32),
                constrained=(np.ones(n, np.uint8) if surface["kind"] != "none" else np.zeros(n, np.uint8))
                if constrained is None else np.ascontiguousarray(constrained, np.uint8))


def sphere_system(n=1000, R=10.0, seed=1, dmin=0.8, precision="fp64", dt=0.001, tol=1e-12,
                  replica=0, interacting=True, **over):
    """Plain-method workload: n WCA particles on a sphere of radius R placed
    uniformly with overlaps closer than dmin rejected, Maxwell velocities at
    kT = 1 (projected on the tangent plane by the library / oracle)."""
    g = rng(seed, 0xFFFFFFFF - replica)
    surf = {"kind": "sphere", "center": (0.0, 0.0, 0.0), "p": (R, 0.0, 0.0, 0.0)}
    x = rsa(lambda k, m: sample_surface(surf, m, g), [n], dmin, g)[0]
    prm = wca_params(precision=precision, dt=dt, rattle_tol=tol, seed=seed, replica=replica, **over)
    if not interacting:
        prm = noninteracting(prm)
    v = maxwell(n, prm["kT"], 1.0, g)
    return _system(f"sphere_N{n}_R{R:g}", surf, prm, x, v)


def free_on_surface(surf: dict, n: int, seed: int = 3, dt: float = 0.002, precision: str = "mixed", box=None):
    """n non-interacting particles sampled uniformly by area on a surface with
    Maxwell velocities at kT = 1 (gamma = m = 1, so D = kT/(m gamma) = 1): the
    inputs of the diffusion laws of SI Section S1.3."""
    prm = noninteracting(wca_params(dt=dt, seed=seed, precision=precision, rattle_tol=1e-10))
    g = np.random.default_rng(seed)
    x = sample_surface(surf, n, g, box=box)
    return [_system("free", surf, prm, x, maxwell(n, 1.0, 1.0, g))]


def c1_plain_sphere():
    """1,000 WCA particles on a sphere R = 10 sigma, float64 path, dt = 0.001,
    RATTLE tolerance 1e-12, seed 1; overlaps rejected below 0.8 sigma
    (phi = 0.787 exceeds the jamming limit of RSA at d0)."""
    return [sphere_system(1000, 10.0, seed=1, dmin=0.8, precision="fp64", dt=0.001, tol=1e-12)]


def ellipsoid_axes_for(n: int, phi: float, base=(150.0, 120.0, 90.0)) -> tuple:
    """Semi-axes of the base ellipsoid's shape scaled to give area fraction phi."""
    A0 = ellipsoid_area(*base, n=600)
    s = math.sqrt(n * A_P / phi / A0)
    return tuple(s * a for a in base)


def c2_ellipsoid_torus(n_ell=200_000, n_tor=50_000, seed=1, dmin=1.0, precision="mixed",
                       dt=0.002, tol=1e-10, torus=(120.0, 40.0)):
    """Mixed-precision workload: n_ell WCA particles at area fraction 0.4 on
    an ellipsoid of the shape (150, 120, 90) sigma (scaled so that the count
    and the fraction both hold: 200,000 particles need semi-axes
    (249.0, 199.2, 149.4) sigma), and n_tor on a torus R = 120, r = 40 sigma
    (phi = 0.261) as a separate system. For smaller n the torus is scaled so
    that its area fraction stays the same."""
    g = rng(seed, 2)
    axes = ellipsoid_axes_for(n_ell, 0.4)
    ell = {"kind": "ellipsoid", "center": (0.0, 0.0, 0.0), "p": (*axes, 0.0)}
    phi_t = 50_000 * A_P / torus_area(*torus)
    s = math.sqrt(n_tor * A_P / phi_t / torus_area(*torus))
    tor = {"kind": "torus", "center": (0.0, 0.0, 0.0), "p": (torus[0] * s, torus[1] * s, 0.0, 0.0)}
    xs = rsa(lambda k, m: sample_surface(ell if k == 0 else tor, m, g), [n_ell, n_tor], dmin, g)
    out = []
    for k, (surf, x) in enumerate(((ell, xs[0]), (tor, xs[1]))):
        prm = wca_params(precision=precision, dt=dt, rattle_tol=tol, seed=seed, replica=k)
        out.append(_system(["ellipsoid", "torus"][k], surf, prm, x, maxwell(x.shape[0], 1.0, 1.0, g)))
    return out


def c3_bump_crowders(n_surf=100_000, n_free=900_000, seed=1, dmin=1.0, precision="mixed",
                     dt=0.002, tol=1e-10, phi_surf=0.4, phi_vol=0.2):
    """Mixed constrained/free workload: n_surf particles on a Gaussian bump
    z = A exp(-rho^2/2w^2) in a periodic square box, plus n_free free
    crowders in a slab between two V_w walls. The stated box (300 sigma,
    A = 20, w = 15) cannot hold 100,000 particles, so box, A and w are
    scaled together to give the surface area fraction phi_surf; the slab
    height follows from the crowders' volume fraction phi_vol with
    v_p = pi d0^3 / 6."""
    L0, A0, w0 = 300.0, 20.0, 15.0
    a0 = bump_area(L0, A0, w0, n=600)
    s = math.sqrt(n_surf * A_P / phi_surf / a0)
    L, A, w = L0 * s, A0 * s, w0 * s
    v_p = math.pi * D0 ** 3 / 6.0
    h = n_free * v_p / phi_vol / (L * L)
    zlo, zhi = -h / 2 - 0.5, A + h / 2 + 0.5
    box = ((-L / 2, -L / 2, zlo - 2.0), (L / 2, L / 2, zhi + 2.0))
    g = rng(seed, 3)
    surf = {"kind": "gaussian_bump", "center": (0.0, 0.0, 0.0), "p": (A, w, 0.0, 0.0)}
    prm = wca_params(precision=precision, dt=dt, rattle_tol=tol, seed=seed, replica=0,
                     box_lo=box[0], box_hi=box[1], periodic=(1, 1, 0), wall_enable=1,
                     wall_lo_z=zlo, wall_hi_z=zhi, wall_eps=1.0, wall_sigma=1.0)
    xs = rsa(lambda k, m: sample_surface(surf, m, g, box=box), [n_surf], dmin, g,
             periodic=(1, 1, 0), box=box)[0]
    wall_rc = D0

    def crowders(k, m):
        xy = np.asarray(box[0][:2]) + g.random((m, 2)) * L
        z = zlo + wall_rc + g.random(m) * (zhi - zlo - 2 * wall_rc)
        return np.column_stack([xy, z])
    xf = rsa(crowders, [n_free], dmin, g, periodic=(1, 1, 0), box=box,
             fixed=xs, fixed_group=np.zeros(n_surf, np.int64))[0]
    x = np.vstack([xs, xf])
    con = np.concatenate([np.ones(n_surf, np.uint8), np.zeros(n_free, np.uint8)])
    return [_system("bump_crowders", surf, prm, x, maxwell(x.shape[0], 1.0, 1.0, g), constrained=con)]


_C4_CHUNK = 256  # replicas per placement chunk (fixed, so results do not depend on workers)


def _c4_chunk(args):
    seed, chunk, Rs, Ns, dmin = args
    g = rng(seed, 0x40000 + chunk)
    Rarr = np.asarray(Rs)

    def on_spheres(groups):
        v = g.standard_normal((groups.shape[0], 3))
        v /= np.linalg.norm(v, axis=1, keepdims=True)
        return v * Rarr[groups][:, None]
    xs = rsa(None, Ns, dmin, g, sampler_multi=on_spheres)
    vs = [maxwell(n, 1.0, 1.0, g) for n in Ns]
    return xs, vs


def c4_replicas(nrep=4096, seed=1, nmin=50, nmax=2000, rmin=5.0, rmax=40.0, phimin=0.05,
                phimax=0.5, dmin=1.0, precision="mixed", dt=0.002, tol=1e-10, workers=None):
    """Batched replicas: nrep independent sphere systems with N ~ U[nmin, nmax]
    and R ~ U[rmin, rmax], redrawn until phi = N A_p / (4 pi R^2) lies in
    [phimin, phimax]; WCA, gamma = kT = 1. Placement runs in chunks of 256
    replicas, each with its own seeded stream (in parallel when workers > 1)."""
    g = rng(seed, 4)
    Ns, Rs = [], []
    while len(Ns) < nrep:
        N = int(g.integers(nmin, nmax + 1))
        R = float(rmin + (rmax - rmin) * g.random())
        phi = N * A_P / (4 * math.pi * R * R)
        if phimin <= phi <= phimax:
            Ns.append(N)
            Rs.append(R)
    jobs = [(seed, c, Rs[c * _C4_CHUNK:(c + 1) * _C4_CHUNK], Ns[c * _C4_CHUNK:(c + 1) * _C4_CHUNK], dmin)
            for c in range((nrep + _C4_CHUNK - 1) // _C4_CHUNK)]
    if workers is None:
        import os
        workers = min(len(jobs), os.cpu_count() or 1)
    if workers > 1 and len(jobs) > 1:
        import concurrent.futures as cf
        import multiprocessing as mp
        with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
            parts = list(ex.map(_c4_chunk, jobs))
    else:
        parts = [_c4_chunk(j) for j in jobs]
    out = []
    k = 0
    for xs, vs in parts:
        for x, v in zip(xs, vs):
            surf = {"kind": "sphere", "center": (0.0, 0.0, 0.0), "p": (Rs[k], 0.0, 0.0, 0.0)}
            prm = wca_params(precision=precision, dt=dt, rattle_tol=tol, seed=seed, replica=k)
            out.append(_system(f"replica{k}", surf, prm, x, v))
            k += 1
    return out


def c5_bead_molecules(nmol=20_000, beads=5, R=60.0, seed=1, dmin=1.0, precision="mixed",
                      dt=0.002, tol=1e-10, bond_k=100.0, bond_r0=1.0):
    """Bead molecules on a spherical template: nmol linear chains of `beads`
    beads (type = bead index), bead 0 held on a sphere of radius R, beads
    1..beads-1 free and placed radially outward at bond_r0 spacing; harmonic
    bonds V = k (r - r0)^2; LJ with eps = 2 and cutoff 2.5 sigma between
    type-3 beads of different molecules, WCA between all other pairs of
    different molecules (pairs within a molecule are excluded)."""
    nt = beads
    prm = wca_params(ntypes=nt, precision=precision, dt=dt, rattle_tol=tol, seed=seed,
                     beads_per_mol=beads, bond_k=bond_k, bond_r0=bond_r0, exclude_intramol=1)
    if nt > 3:
        prm["eps"][3, 3] = 2.0
        prm["rcut"][3, 3] = 2.5
    g = rng(seed, 5)
    surf = {"kind": "sphere", "center": (0.0, 0.0, 0.0), "p": (R, 0.0, 0.0, 0.0)}
    x0 = rsa(lambda k, m: sample_surface(surf, m, g), [nmol], dmin, g)[0]
    u = x0 / np.linalg.norm(x0, axis=1, keepdims=True)
    x = np.empty((nmol, beads, 3))
    for b in range(beads):
        x[:, b, :] = u * (R + b * bond_r0)
    x = x.reshape(-1, 3)
    ext = R + beads * bond_r0 + 10.0
    prm["box_lo"] = (-ext, -ext, -ext)
    prm["box_hi"] = (ext, ext, ext)
    type_ = np.tile(np.arange(beads, dtype=np.int32), nmol)
    con = (type_ == 0).astype(np.uint8)
    return [_system("bead_molecules", surf, prm, x, maxwell(x.shape[0], 1.0, 1.0, g),
                    type_=type_, constrained=con)]


def nve_systems(pair_form: int, n: int = 500, phi: float = 0.3, seed: int = 1, precision: str = "fp64",
                dt: float = 0.0005, tol: float = 1e-12, rc: float = 2.5, dmin: float = 1.0):
    """Energy-conservation workload of the SI: n Lennard-Jones particles
    (eps = sigma = m = 1, cutoff rc, truncated-shifted (pair_form 0) or
    linearly smoothed (1)) held on a sphere, a cylinder (periodic along its
    axis), a torus and a plane (periodic in x and y), each at area fraction
    phi, gamma = 0 (constant energy), Maxwell velocities at kT = 1. Returns
    the four systems (one batch)."""
    area = n * A_P / phi
    out = []
    specs = []
    R_s = math.sqrt(area / (4 * math.pi))
    specs.append(("sphere", {"kind": "sphere", "center": (0.0, 0.0, 0.0), "p": (R_s, 0, 0, 0)}, {}))
    R_c = 6.0
    L_c = area / (2 * math.pi * R_c)
    specs.append(("cylinder", {"kind": "cylinder", "center": (0.0, 0.0, 0.0), "p": (R_c, 2.0, 0, 0)},
                  dict(box_lo=(-R_c - 3, -R_c - 3, -L_c / 2), box_hi=(R_c + 3, R_c + 3, L_c / 2),
                       periodic=(0, 0, 1))))
    r_t = 3.0
    R_t = area / (4 * math.pi ** 2 * r_t)
    specs.append(("torus", {"kind": "torus", "center": (0.0, 0.0, 0.0), "p": (R_t, r_t, 0, 0)}, {}))
    L_p = math.sqrt(area)
    specs.append(("plane", {"kind": "plane", "center": (0.0, 0.0, 0.0), "p": (0.0, 0.0, 1.0, 0)},
                  dict(box_lo=(-L_p / 2, -L_p / 2, -3.0), box_hi=(L_p / 2, L_p / 2, 3.0), periodic=(1, 1, 0))))
    for k, (name, surf, extra) in enumerate(specs):
        prm = wca_params(precision=precision, dt=dt, rattle_tol=tol, gamma=0.0, seed=seed, replica=k,
                         pair_form=pair_form, **extra)
        prm["rcut"][0, 0] = rc
        g = rng(seed, 100 + k)
        box = (prm["box_lo"], prm["box_hi"]) if extra else None
        x = rsa(lambda kk, m: sample_surface(surf, m, g, box=box), [n], dmin, g, periodic=prm["periodic"],
                box=box)[0]
        out.append(_system(name, surf, prm, x, maxwell(n, 1.0, 1.0, g)))
    return out


def lj_lattice(k: int = 46, a: float = 1.0833, rc: float = 2.5, seed: int = 3, precision: str = "mixed",
               dt: float = 0.001, tol: float = 1e-10, jitter: float = 0.06) -> list:
    """Dense free Lennard-Jones liquid (a stress case of the pair kernel, not
    a workload of the paper): k^3 particles on a simple cubic lattice of
    spacing a (density 1/a^3, 0.79 at a = 1.0833) moved by uniform jitter of
    +-jitter, in a periodic cube of edge k a, cutoff rc, no surface."""
    L = k * a
    g = rng(seed, 21)
    idx = np.stack(np.meshgrid(*[np.arange(k)] * 3, indexing="ij"), -1).reshape(-1, 3)
    x = (idx + 0.5) * a + g.uniform(-jitter, jitter, idx.shape) - L / 2
    prm = wca_params(precision=precision, dt=dt, rattle_tol=tol, seed=seed,
                     box_lo=(-L / 2,) * 3, box_hi=(L / 2,) * 3, periodic=(1, 1, 1))
    prm["rcut"][0, 0] = rc
    surf = {"kind": "none", "center": (0.0, 0.0, 0.0), "p": (0.0, 0.0, 0.0, 0.0)}
    return [_system("lj_lattice", surf, prm, x, maxwell(x.shape[0], 1.0, 1.0, g))]


def capsid_systems(nsys: int = 1, ncone: int = 60, sigma3: float = 1.75, seed: int = 1, precision: str = "mixed",
                   dt: float = 0.002, tol: float = 1e-10, dmin: float = 1.8, phi_base: float = 0.45):
    """Capsomere (cone) self-assembly on a spherical template, the capsid model
    of SI S3.2: ncone cones of four beads (types 0..3 with sizes sigma_i =
    1, 1.35, sigma3, 1), additive mixing sigma_ij = (sigma_i + sigma_j)/2,
    well depth 4 kT, cutoff 4 sigma_0 between like beads of types 1 and 2
    (the SI's types 2 and 3) and 2^(1/6) sigma_ij (purely repulsive) for
    every other pair, Lennard-Jones only between different cones; masses
    proportional to the bead volume; bonds k = 50 kT/sigma_0^2 with rest
    lengths 2^(1/6)(sigma_i + sigma_j)/4; bend angles k_a = 250 kT/rad^2,
    theta0 = pi; the first bead of each cone held on the sphere, the others
    free; a repulsive spherical wall (eps_w = sigma_w = 1) at R - 1 keeps
    free beads out of the sphere. The sphere radius follows from the base
    beads' area fraction phi_base; cones start straight and radial with
    their bases placed by random sequential addition at distance >= dmin.
    Returns nsys independently seeded systems (one batch)."""
    sig = np.array([1.0, 1.35, sigma3, 1.0])
    nt = 4
    sij = 0.5 * (sig[:, None] + sig[None, :])
    eps = np.full((nt, nt), 4.0)
    rc = 2 ** (1 / 6) * sij
    rc[1, 1] = 4.0
    rc[2, 2] = 4.0
    r0 = 2 ** (1 / 6) * sij / 2
    R = math.sqrt(ncone * math.pi * (dmin / 2) ** 2 / phi_base / (4 * math.pi))
    ext = R + r0[0, 1] + r0[1, 2] + r0[2, 3] + 6.0
    out = []
    for s in range(nsys):
        prm = wca_params(ntypes=nt, precision=precision, dt=dt, rattle_tol=tol, seed=seed, replica=s,
                         mass=list(sig ** 3), beads_per_mol=4, bond_k=50.0, bond_r0=0.0, bond_r0_mix=1,
                         angle_k=250.0, angle_theta0=math.pi, exclude_intramol=1, wall_enable=1, wall_kind=1,
                         wall_radius=R - 1.0, wall_center=(0.0, 0.0, 0.0), wall_eps=1.0, wall_sigma=1.0,
                         box_lo=(-ext, -ext, -ext), box_hi=(ext, ext, ext))
        prm["sigma"], prm["eps"], prm["rcut"] = sij.copy(), eps.copy(), rc.copy()
        g = rng(seed, 1000 + s)
        surf = {"kind": "sphere", "center": (0.0, 0.0, 0.0), "p": (R, 0.0, 0.0, 0.0)}
        base = rsa(lambda k, m: sample_surface(surf, m, g), [ncone], dmin, g)[0]
        u = base / np.linalg.norm(base, axis=1, keepdims=True)
        radii = R + np.concatenate([[0.0], np.cumsum([r0[0, 1], r0[1, 2], r0[2, 3]])])
        x = (u[:, None, :] * radii[None, :, None]).reshape(-1, 3)
        type_ = np.tile(np.arange(4, dtype=np.int32), ncone)
        con = (type_ == 0).astype(np.uint8)
        out.append(_system("capsid", surf, prm, x, maxwell(x.shape[0], 1.0, np.asarray(prm["mass"])[type_], g),
                           type_=type_, constrained=con))
    return out


def sphere_and_plane2d(n: int = 1_000_000, phi: float = 0.4, seed: int = 1, precision: str = "mixed",
                       dt: float = 0.002, tol: float = 1e-10, dmin: float = 1.0):
    """The performance comparison of Section 3.1 at equal density: n WCA
    particles held on a sphere by RATTLE, and n WCA particles in a periodic
    2D plane of the same area with no constraint (surface kind xy2d: the z
    updates are not evaluated), both at area fraction phi, kT = gamma = 1.
    Returns (sphere systems, plane systems), one system each."""
    area = n * A_P / phi
    R = math.sqrt(area / (4 * math.pi))
    g = rng(seed, 300)
    prm = wca_params(precision=precision, dt=dt, rattle_tol=tol, seed=seed)
    surf = {"kind": "sphere", "center": (0.0, 0.0, 0.0), "p": (R, 0, 0, 0)}
    x = rsa(lambda k, m: sample_surface(surf, m, g), [n], dmin, g)[0]
    sphere = [_system("sphere", surf, prm, x, maxwell(n, 1.0, 1.0, g))]
    L = math.sqrt(area)
    prm2 = wca_params(precision=precision, dt=dt, rattle_tol=tol, seed=seed, box_lo=(-L / 2, -L / 2, -1.0),
                      box_hi=(L / 2, L / 2, 1.0), periodic=(1, 1, 0))
    flat = {"kind": "xy2d", "center": (0.0, 0.0, 0.0), "p": (0, 0, 0, 0)}
    box = (prm2["box_lo"], prm2["box_hi"])
    x2 = rsa(lambda k, m: sample_surface(flat, m, g, box=box), [n], dmin, g, periodic=prm2["periodic"], box=box)[0]
    v2 = maxwell(n, 1.0, 1.0, g)
    v2[:, 2] = 0.0
    plane = [_system("plane2d", flat, prm2, x2, v2, constrained=np.zeros(n, np.uint8))]
    return sphere, plane


THYLAKOID_SI = dict(Lx=15.0, Lz=30.0, Rc=3.0, Lb=10.0)  # the SI's surface parameters (R = R_c = 3)


def thylakoid_surface(Rb: float = 1.5, Lx: float = 15.0, Rc: float = 3.0, Lb: float = 10.0,
                      center=(0.0, 0.0, 0.0)) -> dict:
    """The thylakoid composite of SI S3.1 (two rounded-square blocks joined by
    a bridge of radius Rb through toroidal connectors; z is periodic)."""
    return {"kind": "thylakoid", "center": tuple(center), "p": (Rb, Lx, Rc, Lb)}


def thylakoid_area_parts(Rb, Lx, Rc, Lb, Lz):
    """Areas of the pieces: the planes of both blocks (the two face planes
    without their connector holes), the corner cylinders, the bridge and the
    two connectors (SI S3.1: A_conn = pi R^2 (pi - 2) + pi^2 R R_b with R = R_c)."""
    a_planes = 8 * Lx * Lz - 2 * math.pi * (Rb + Rc) ** 2
    a_corners = 2 * 2 * math.pi * Rc * Lz
    a_bridge = 2 * math.pi * Rb * Lb
    a_conn = math.pi * Rc ** 2 * (math.pi - 2) + math.pi ** 2 * Rc * Rb
    return dict(planes=a_planes, corners=a_corners, bridge=a_bridge, connectors=2 * a_conn)


def sample_thylakoid(surf: dict, n: int, g: np.random.Generator, Lz: float) -> np.ndarray:
    """n points uniform in area on the thylakoid composite (z in [c_z - Lz/2,
    c_z + Lz/2))."""
    Rb, Lx, Rc, Lb = surf["p"]
    xc, yc, zc = surf["center"]
    x0L, x0R = xc - Lb / 2, xc + Lb / 2
    xfL, xfR = x0L - Rc, x0R + Rc
    parts = thylakoid_area_parts(Rb, Lx, Rc, Lb, Lz)
    names = list(parts)
    w = np.array([parts[k] for k in names])
    which = g.choice(len(names), size=n, p=w / w.sum())
    out = np.empty((n, 3))
    for kk, name in enumerate(names):
        idx = np.flatnonzero(which == kk)
        m = idx.size
        if m == 0:
            continue
        z = zc - Lz / 2 + g.random(m) * Lz
        if name == "bridge":
            ph = g.random(m) * 2 * math.pi
            out[idx] = np.column_stack([x0L + g.random(m) * Lb, yc + Rb * np.cos(ph), zc + Rb * np.sin(ph)])
        elif name == "connectors":
            pts = []
            while len(pts) < m:
                k = 2 * (m - len(pts)) + 16
                al = g.random(k) * math.pi / 2
                r = Rb + Rc - Rc * np.cos(al)
                keep = g.random(k) < r / (Rb + Rc)
                al, r = al[keep], r[keep]
                side = g.random(al.size) < 0.5
                xx = np.where(side, x0L - Rc * np.sin(al), x0R + Rc * np.sin(al))
                ph = g.random(al.size) * 2 * math.pi
                pts.extend(np.column_stack([xx, yc + r * np.cos(ph), zc + r * np.sin(ph)]))
            out[idx] = np.array(pts[:m])
        elif name == "corners":
            blk = g.random(m) < 0.5
            cor = g.integers(0, 4, m)
            ixl = np.where(blk, xfL - Rc - Lx, xfR + Rc)
            cx = ixl + np.where(cor % 2 == 1, Lx, 0.0)
            cy = yc + np.where(cor // 2 == 1, Lx / 2, -Lx / 2)
            base = np.where(cor % 2 == 1, 0.0, math.pi)  # quarter facing outward in x
            sgn = np.where(cor // 2 == 1, 1.0, -1.0)
            a = g.random(m) * math.pi / 2
            # the quarter between the outward x direction and the outward y direction
            ang = np.where(cor % 2 == 1, sgn * a, math.pi - sgn * a)
            del base
            out[idx] = np.column_stack([cx + Rc * np.cos(ang), cy + Rc * np.sin(ang), z])
        else:  # planes: 4 per block; the face planes lose the connector holes
            pts = []
            while len(pts) < m:
                k = 2 * (m - len(pts)) + 16
                blk = g.random(k) < 0.5
                side = g.integers(0, 4, k)
                t = g.random(k) * Lx - Lx / 2
                zz = zc - Lz / 2 + g.random(k) * Lz
                ixl = np.where(blk, xfL - Rc - Lx, xfR + Rc)
                ixh = ixl + Lx
                xs = np.where(side == 0, ixl - Rc, np.where(side == 1, ixh + Rc, (ixl + ixh) / 2 + t))
                ys = np.where(side < 2, yc + t, np.where(side == 2, yc - Lx / 2 - Rc, yc + Lx / 2 + Rc))
                dz = zz - zc
                hole = (np.abs(xs - np.where(blk, xfL, xfR)) < 1e-12) & (np.hypot(ys - yc, dz) < Rb + Rc)
                ok = ~hole
                pts.extend(np.column_stack([xs[ok], ys[ok], zz[ok]]))
            out[idx] = np.array(pts[:m])
    return out


def thylakoid_system(n: int = 3000, Rb: float = 1.5, phi: float = None, seed: int = 1, precision: str = "mixed",
                     dt: float = 0.002, tol: float = 1e-10, dmin: float = 1.0, interacting: bool = True):
    """Crowded diffusion on the thylakoid composite of SI S3.1 with its surface
    parameters (L_x = 15, L_z = 30, R_c = R = 3, L_b = 10, bridge radius Rb):
    n WCA particles (the SI uses 2000-4000) placed by random sequential
    addition, periodic z of length L_z, kT = gamma = 1. (phi is ignored; the
    area fraction follows from n.)"""
    surf = thylakoid_surface(Rb, THYLAKOID_SI["Lx"], THYLAKOID_SI["Rc"], THYLAKOID_SI["Lb"])
    Lz = THYLAKOID_SI["Lz"]
    w = THYLAKOID_SI["Lx"] + 2 * THYLAKOID_SI["Rc"]
    ext_x = THYLAKOID_SI["Lb"] / 2 + THYLAKOID_SI["Rc"] + w + 3.0
    prm = wca_params(precision=precision, dt=dt, rattle_tol=tol, seed=seed,
                     box_lo=(-ext_x, -w / 2 - 3.0, -Lz / 2), box_hi=(ext_x, w / 2 + 3.0, Lz / 2),
                     periodic=(0, 0, 1))
    if not interacting:
        prm = noninteracting(prm)
    g = rng(seed, 400)
    box = (prm["box_lo"], prm["box_hi"])
    if interacting:
        x = rsa(lambda k, m: sample_thylakoid(surf, m, g, Lz), [n], dmin, g, periodic=prm["periodic"], box=box)[0]
    else:  # free particles may overlap
        x = sample_thylakoid(surf, n, g, Lz)
    return [_system("thylakoid", surf, prm, x, maxwell(n, 1.0, 1.0, g))]
