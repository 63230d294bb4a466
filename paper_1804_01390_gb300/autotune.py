"""Kernel-variant autotuning with an on-disk cache.

The library times its interior-kernel variants on a live context (``pml_autotune``).
This module keys the winner by (device name, dimension, precision, box shape, layer
width) and keeps it in a JSON file (``$PML_AUTOTUNE_CACHE`` or
``~/.cache/pml_autotune.json``) so later contexts of the same shape skip the timing.
"""
from __future__ import annotations

import json
import os

from . import _lib


def cache_path() -> str:
    return os.environ.get("PML_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "pml_autotune.json"))


def _key(solver) -> str:
    import torch
    name = torch.cuda.get_device_name(solver.device)
    return "%s|%dd|fp%d|%s|w%d" % (name, solver.ndim, solver.precision,
                                   "x".join(str(t) for t in solver.T), solver.w)


def _load() -> dict:
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except Exception:
        return {}


def tune(solver, steps: int = 20, use_cache: bool = True):
    """Select the fastest interior-kernel variant for this solver's shape.

    Advances the solver's state (tune before ``set_initial``).  Returns
    (variant, {variant: ms per step} or None when the cached choice was used).
    """
    key = _key(solver)
    cache = _load() if use_cache else {}
    if key in cache:
        _lib.pml_set_variant(solver.ctx, int(cache[key]["variant"]))
        return int(cache[key]["variant"]), None
    chosen, times = _lib.pml_autotune(solver.ctx, steps)
    table = {int(i): float(t) for i, t in enumerate(times)}
    cache[key] = {"variant": chosen, "ms_per_step": table}
    try:
        os.makedirs(os.path.dirname(cache_path()), exist_ok=True)
        tmp = cache_path() + ".tmp%d" % os.getpid()
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
        os.replace(tmp, cache_path())
    except OSError:
        pass
    return chosen, table
