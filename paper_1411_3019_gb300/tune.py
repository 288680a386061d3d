"""Autotuner of the step's launch options.

For a handle with a state, times the step under each candidate setting and
applies the fastest:

* the global engine (one graph of five kernels per step) with every
  combination of the pair kernel's visiting order and lanes per particle,
  and with the cell-tiled pair kernel at 32, 16 and 8 particles per warp
  where the grid allows it, one step per
  trial after an L2 flush (as the benchmark times it);
* the resident engine (one persistent launch, one CTA per system), if the
  systems fit it, for several CTA sizes, a run of `resident_steps` steps per
  trial (its cost per step, with its one cell-list rebuild per call spread
  over the run).

With the Verlet list (`autotune_list`): the skin, which sets the cell size
r_c + skin of a new handle, and the list walk's particles per warp, each
timed over a run of steps that includes the rebuilds the skin causes.

The visiting order and the resident engine change no bit of the results;
the lanes per particle and the cell-tiled kernel add each particle's pair
terms in another order, so their forces differ from the default's by float
rounding only. The choice can be cached in a JSON file keyed by a
caller-given GPU name and the workload's shape (particles, systems), so
later runs skip the trials.
"""
from __future__ import annotations

import itertools
import json
import os

from . import md

GLOBAL_OPTIONS = {md.MD_OPT_PAIR_ORDER: (1, 0), md.MD_OPT_PAIR_LANES: (1, 2, 4)}
RESIDENT_THREADS = (0, 256, 128)  # 0: chosen per size class
TILE_SLOTS = (32, 16, 8)  # particles per warp of the cell-tiled pair kernel
NAMES = {md.MD_OPT_PAIR_ORDER: "pair_order", md.MD_OPT_PAIR_LANES: "pair_lanes", md.MD_OPT_ENGINE: "engine",
         md.MD_OPT_RESIDENT_THREADS: "resident_threads", md.MD_OPT_PAIR_TILE: "pair_tile"}


def _key(h, gpu_name: str) -> str:
    info = md.md_info(h)
    return f"{gpu_name}|n={info['n']}|nsys={info['nsys']}"


def candidates(h):
    """Option settings to try: the global engine's combinations, then the
    resident engine's CTA sizes if the handle's systems fit it."""
    out = []
    opts = list(GLOBAL_OPTIONS)
    for combo in itertools.product(*(GLOBAL_OPTIONS[o] for o in opts)):
        out.append({md.MD_OPT_ENGINE: 0, md.MD_OPT_PAIR_TILE: 0, **dict(zip(opts, combo))})
    md.md_set_option(h, md.MD_OPT_ENGINE, 0)
    try:
        md.md_set_option(h, md.MD_OPT_PAIR_TILE, TILE_SLOTS[0])
        out.extend({md.MD_OPT_ENGINE: 0, md.MD_OPT_PAIR_TILE: t} for t in TILE_SLOTS)
    except md.MdError:
        pass  # buckets are hashed: no cell-tiled kernel
    finally:
        md.md_set_option(h, md.MD_OPT_PAIR_TILE, 0)
    for thr in RESIDENT_THREADS:
        try:
            md.md_set_option(h, md.MD_OPT_RESIDENT_THREADS, thr)
            md.md_set_option(h, md.MD_OPT_ENGINE, 1)
        except md.MdError:
            continue
        finally:
            md.md_set_option(h, md.MD_OPT_ENGINE, 0)
        out.append({md.MD_OPT_ENGINE: 1, md.MD_OPT_RESIDENT_THREADS: thr})
    return out


def apply(h, setting: dict) -> None:
    md.md_set_option(h, md.MD_OPT_ENGINE, 0)
    md.md_set_option(h, md.MD_OPT_PAIR_TILE, 0)
    for opt, val in setting.items():
        if opt != md.MD_OPT_ENGINE:
            md.md_set_option(h, opt, val)
    md.md_set_option(h, md.MD_OPT_ENGINE, setting.get(md.MD_OPT_ENGINE, 0))


def time_setting(h, setting: dict, trials: int, flush, resident_steps: int) -> float:
    """Mean milliseconds per step of one setting."""
    apply(h, setting)
    steps = resident_steps if setting.get(md.MD_OPT_ENGINE, 0) == 1 else 1
    md.md_profile_step(h, steps)  # warm this configuration
    total = 0.0
    for _ in range(trials):
        if flush is not None:
            flush()
        total += sum(md.md_profile_step(h, steps).values())
    return total / trials


def autotune(h, trials: int = 3, flush=None, cache: str | None = None, gpu_name: str = "gpu",
             resident_steps: int = 32):
    """Try every candidate setting on handle h; apply and return the best.
    The trial steps advance the handle's state."""
    key = _key(h, gpu_name)
    if cache and os.path.exists(cache):
        with open(cache) as fh:
            known = json.load(fh)
        if key in known:
            best = {int(k): v for k, v in known[key]["options"].items()}
            apply(h, best)
            return {"cached": True, "options": {NAMES[k]: v for k, v in best.items()}}
    results = [(time_setting(h, c, trials, flush, resident_steps), c) for c in candidates(h)]
    results.sort(key=lambda r: r[0])
    best_ms, best = results[0]
    apply(h, best)
    if cache:
        known = {}
        if os.path.exists(cache):
            with open(cache) as fh:
                known = json.load(fh)
        known[key] = {"options": {str(k): v for k, v in best.items()}, "ms": best_ms}
        with open(cache, "w") as fh:
            json.dump(known, fh, indent=1)
    return {"cached": False, "best_ms": best_ms, "options": {NAMES[k]: v for k, v in best.items()},
            "trials": [{"ms": ms, **{NAMES[k]: v for k, v in c.items()}} for ms, c in results]}


LIST_SKINS = (0.3, 0.4, 0.5, 0.6)
LIST_WARPS = (32, 16)
LIST_NAMES = {md.MD_OPT_LIST_WARP: "list_warp"}


def _with_cell_size(systems, skin: float):
    """Copies of the system dicts with the cell edge r_c + skin (the list's
    reach), the cell size a handle with that skin needs."""
    out = []
    for sy in systems:
        rc = float(max(map(max, sy["params"]["rcut"])))
        out.append(dict(sy, params=dict(sy["params"], cell_size=rc + skin)))
    return out


def autotune_list(systems, max_neighbors: int, skins=LIST_SKINS, list_warps=LIST_WARPS, steps: int = 100,
                  warmup: int = 20, flush=None, stream=None):
    """Verlet-list step form: the skin (hence the cell size r_c + skin, fixed
    when a handle is created) and the list walk's particles per warp. For
    each skin a handle of the systems is created with that cell size; each
    setting is timed as the sum of the step kernels' mean times over `steps`
    steps (which include the list rebuilds that skin causes), after `warmup`
    steps and an optional L2 flush. Returns the best setting and the trials;
    the handles are destroyed (the caller creates its own with the choice).
    Skins whose list overflows max_neighbors are skipped."""
    trials = []
    if systems and systems[0]["params"].get("precision") in ("fp64", 0):
        list_warps = list_warps[:1]  # the float64 path walks per lane: no warp width to choose
    for skin in skins:
        sim = md.Simulation(_with_cell_size(systems, skin), stream=stream)
        try:
            md.md_set_neighbor_list(sim.h, skin, max_neighbors)
            sim.set_state()
            sim.step(warmup)
            sim.sync()
            for lw in list_warps:
                try:
                    md.md_set_option(sim.h, md.MD_OPT_LIST_WARP, lw)
                except md.MdError:
                    continue  # the float64 path has no warp-queued walk
                md.md_profile_step(sim.h, 2)  # capture and warm this setting
                if flush is not None:
                    flush()
                b0 = md.md_get_option(sim.h, md.MD_OPT_NLIST_BUILDS)
                ms = sum(md.md_profile_step(sim.h, steps).values())
                builds = md.md_get_option(sim.h, md.MD_OPT_NLIST_BUILDS) - b0
                trials.append({"ms": ms, "skin": skin, "list_warp": lw, "builds": int(builds), "steps": steps})
        except md.MdError:
            pass  # e.g. the list is too small at this skin
        finally:
            sim.close()
    if not trials:
        return None
    trials.sort(key=lambda t: t["ms"])
    best = trials[0]
    return {"skin": best["skin"], "list_warp": best["list_warp"], "best_ms": best["ms"], "trials": trials}
