"""Kernel-variant autotuning with an on-disk cache.

The library times its interior-kernel variants (one-step shapes and, for 2D FP32, the
two-step temporally blocked shapes) on a live context (``pml_autotune``).
This module keys the winner by (device name, dimension, precision, box shape, layer
width, number of variants the library offers) and keeps it in a JSON file
(``$PML_AUTOTUNE_CACHE`` or ``~/.cache/pml_autotune.json``) so later contexts of the same
shape skip the timing.  A cached choice the library rejects (a build with other variants)
is timed again.
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
    nvar = _lib.pml_get_variant(solver.ctx)[1]
    return "%s|%dd|fp%d|%s|w%d|n%d" % (name, solver.ndim, solver.precision,
                                       "x".join(str(t) for t in solver.T), solver.w, nvar)


def _load() -> dict:
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except Exception:
        return {}


def select(ctx, variant: int, one_step: int | None = None) -> None:
    """Select `variant`; with a two-step variant, `one_step` (if given) is the one-step
    variant kept for single steps and the adjoint."""
    if one_step is not None and one_step != variant:
        _lib.pml_set_variant(ctx, int(one_step))
    _lib.pml_set_variant(ctx, int(variant))


def _best_one_step(ctx, times) -> int:
    """Fastest variant among those that advance one step per pass (leaves it selected)."""
    best, best_t = 0, float("inf")
    for v, t in enumerate(times):
        _lib.pml_set_variant(ctx, v)
        if _lib.pml_get_time_block(ctx) == 1 and t < best_t:
            best, best_t = v, t
    return best


def tune(solver, steps: int = 20, use_cache: bool = True):
    """Select the fastest interior-kernel variant for this solver's shape.

    Advances the solver's state (tune before ``set_initial``).  Returns
    (variant, {variant: ms per step} or None when the cached choice was used); the
    fastest one-step variant (for single steps and the adjoint) is in
    ``solver.one_step_variant``.
    """
    key = _key(solver)
    cache = _load() if use_cache else {}
    if key in cache:
        rec = cache[key]
        one = int(rec.get("one_step", rec["variant"]))
        try:
            select(solver.ctx, int(rec["variant"]), one)
            solver.one_step_variant = one
            return int(rec["variant"]), None
        except _lib.PMLError:
            pass   # not a variant of this build: time them again
    chosen, times = _lib.pml_autotune(solver.ctx, steps)
    one = _best_one_step(solver.ctx, times)
    select(solver.ctx, chosen, one)
    solver.one_step_variant = one
    table = {int(i): float(t) for i, t in enumerate(times)}
    cache[key] = {"variant": chosen, "one_step": one, "ms_per_step": table}
    try:
        os.makedirs(os.path.dirname(cache_path()), exist_ok=True)
        tmp = cache_path() + ".tmp%d" % os.getpid()
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
        os.replace(tmp, cache_path())
    except OSError:
        pass
    return chosen, table
