"""Autotuner of the step's launch options.

For a handle with a state, times one step (every kernel, CUDA events, L2
flushed between trials when a flush buffer is given) under each combination
of the tunable options -- the visiting order of the pair kernel and the lanes
per particle -- applies the fastest and returns the measurements. The choice
can be cached in a JSON file keyed by a caller-given GPU name and the workload's
shape (particles, systems), so later runs skip the trials.
"""
from __future__ import annotations

import itertools
import json
import os

from . import md

OPTIONS = {
    md.MD_OPT_PAIR_ORDER: (1, 0),
    md.MD_OPT_PAIR_LANES: (1, 2, 4),
}
NAMES = {md.MD_OPT_PAIR_ORDER: "pair_order", md.MD_OPT_PAIR_LANES: "pair_lanes"}


def _key(h, gpu_name: str) -> str:
    info = md.md_info(h)
    return f"{gpu_name}|n={info['n']}|nsys={info['nsys']}"


def autotune(h, trials: int = 3, flush=None, cache: str | None = None, gpu_name: str = "gpu"):
    """Try every option combination on handle h; apply and return the best."""
    key = _key(h, gpu_name)
    if cache and os.path.exists(cache):
        with open(cache) as fh:
            known = json.load(fh)
        if key in known:
            best = {int(k): v for k, v in known[key]["options"].items()}
            for opt, val in best.items():
                md.md_set_option(h, opt, val)
            return {"cached": True, "options": {NAMES[k]: v for k, v in best.items()}}
    results = []
    opts = list(OPTIONS)
    for combo in itertools.product(*(OPTIONS[o] for o in opts)):
        for opt, val in zip(opts, combo):
            md.md_set_option(h, opt, val)
        md.md_profile_step(h, 1)  # warm this configuration
        total = 0.0
        for _ in range(trials):
            if flush is not None:
                flush()
            total += sum(md.md_profile_step(h, 1).values())
        results.append((total / trials, dict(zip(opts, combo))))
    results.sort(key=lambda r: r[0])
    best_ms, best = results[0]
    for opt, val in best.items():
        md.md_set_option(h, opt, val)
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
