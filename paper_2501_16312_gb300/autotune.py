"""Autotuner for the rasterizer's launch parameters.

The tuning knobs (sort mode and radix digit width, tile edge, pixels per
blend thread, records per shared-memory batch, resident blend blocks per SM,
one- or two-pass backward chain, and the number of contributing lanes up to
which a backward warp lets each lane add its own colour terms) change only the
schedule: every setting renders bit-identical images (the chain's split and
the backward's reduction form only reorder floating-point sums of
gradients).  The tuner times forward + backward of the caller's own workload
with the library's per-stage CUDA events.  It settles the knobs one group at
a time, each judged on the stages it affects: the sort mode and digit width
on the sort stages; the tile edge and blend schedule on the sort and blend
stages (the tile edge sets the tile-list length as well as the blend's work),
then the sort knobs once more at the chosen edge;
the chain form on the chain stage and the lane threshold on the backward
blend, and the tile order on the range and blend stages (its kernels run
with the ranges).  The choice is cached as JSON keyed by GPU name, primitive kind and
size buckets of the workload.
"""
from __future__ import annotations

import itertools
import json
import math
import os
from typing import Optional

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "linprim_gb300_tuning.json")

SORT_STAGES = ("scan_emit", "sort", "ranges")
BLEND_STAGES = ("blend_fwd", "blend_bwd")


def _bucket(x: float) -> int:
    return int(round(math.log2(max(1.0, x))))


def cache_key(gpu_name: str, kind: int, n_prims: int, cameras) -> str:
    pixels = sum(c.width * c.height for c in cameras)
    return f"{gpu_name}|kind{kind}|n2^{_bucket(n_prims)}|px2^{_bucket(pixels)}|cams{len(cameras)}"


def _time(rast, prims, cameras, bg, dL, grads, images, reps: int):
    import torch
    acc = {}
    for it in range(reps + 1):
        rast.forward(prims, cameras, bg, images=images)
        rast.backward(dL, grads=grads)
        torch.cuda.synchronize()
        t = rast.stage_times()
        if it > 0:   # first repetition warms caches and sizes workspace
            for k, v in t.items():
                acc[k] = acc.get(k, 0.0) + v / reps
    return acc


# (tile edge, pixels per thread) pairs the blends are built for, as the
# library's lp_set_tuning accepts them
TILE_PIX = ((8, 1), (8, 2), (16, 2), (16, 4), (32, 2), (32, 4))

# The search: each group of knobs, its candidates, and the stages it is
# judged on.  Later groups are timed at the earlier groups' choices.  The sort
# knobs are settled twice: first at the starting tile edge, so that the tile
# group compares edges with a sensible sort, then again at the chosen edge
# (the key width, and with it the best digit width, depends on the edge).
_SORT_GROUP = (("sort_mode", "radix_bits", "onesweep"), tuple(itertools.product((0, 1, 2), (4, 6, 8, 11), (0, 1))),
               SORT_STAGES)
GROUPS = (
    _SORT_GROUP,
    (("tile", "pixels_per_thread", "batch", "blocks_per_sm"),
     tuple((t, p, b, 0) for (t, p), b in itertools.product(TILE_PIX, (32, 64, 128))), SORT_STAGES + BLEND_STAGES),
    _SORT_GROUP,
    (("chain_split",), ((0,), (1,)), ("chain",)),
    (("tile_order",), ((0,), (1,)), ("ranges",) + BLEND_STAGES),
)


def search(apply, measure, base: dict) -> dict:
    """Coordinate search over GROUPS.  apply(settings) sets knob values (a
    dict); measure() returns the stage times in ms of one timed forward +
    backward at the current settings.  Returns the choice (base updated with
    the winners, which are left applied), each group's best summed time and
    every trial."""
    choice = dict(base)
    best_ms, results = {}, []
    for names, candidates, stages in GROUPS:
        times = {}
        for values in candidates:
            setting = dict(zip(names, values))
            apply(setting)
            t = measure()
            times[values] = sum(t[s] for s in stages)
            results.append({**setting, **t})
        win = min(times, key=times.get)      # the first candidate wins ties
        choice.update(zip(names, win))
        apply(dict(zip(names, win)))         # later groups are timed at this choice
        label = "+".join(names)
        best_ms[label + " (again)" if label in best_ms else label] = times[win]
    return {"tuning": choice, "best_ms": best_ms, "trials": results}


def load_cache(cache: Optional[str], key: str, knobs=None) -> Optional[dict]:
    """The cached entry for key, or None (missing or unreadable file, or an
    entry whose tuning names other knobs than `knobs`, e.g. one written by a
    build with a different set of knobs)."""
    if not cache or not os.path.exists(cache):
        return None
    try:
        with open(cache) as f:
            entry = json.load(f).get(key)
    except (OSError, ValueError, AttributeError):
        return None
    if entry is None or not isinstance(entry.get("tuning"), dict):
        return None
    if knobs is not None and set(entry["tuning"]) != set(knobs):
        return None
    return entry


def store_cache(cache: Optional[str], key: str, entry: dict) -> None:
    """Adds entry under key, replacing the file atomically; errors are ignored
    (the cache is an optimisation)."""
    if not cache:
        return
    try:
        os.makedirs(os.path.dirname(cache) or ".", exist_ok=True)
        known = {}
        if os.path.exists(cache):
            try:
                with open(cache) as f:
                    known = json.load(f)
            except ValueError:
                known = {}
        known[key] = entry
        with open(cache + ".tmp", "w") as f:
            json.dump(known, f, indent=1)
        os.replace(cache + ".tmp", cache)
    except OSError:
        pass


def tune(rast, prims, cameras, bg=(0.0, 0.0, 0.0), dL=None, reps: int = 3,
         cache: Optional[str] = DEFAULT_CACHE, force: bool = False) -> dict:
    """Pick and apply the fastest tuning for this workload; returns the entry
    (its "tuning" is the choice, now set on rast)."""
    import torch
    gpu = torch.cuda.get_device_name(rast.device)
    key = cache_key(gpu, prims.kind, prims.n, cameras)
    if not force:
        known = load_cache(cache, key, knobs=rast.tuning())
        if known is not None:
            rast.set_tuning(**known["tuning"])
            return known
    P = sum(c.width * c.height for c in cameras)
    images = torch.empty(3 * P, device=rast.device)
    if dL is None:
        dL = torch.ones(3 * P, device=rast.device)
    grads = dict(centre=torch.empty_like(prims.centre), verts=torch.empty_like(prims.verts),
                 opacity=torch.empty_like(prims.opacity), sh=torch.empty_like(prims.sh))
    was_timing = rast.timing()
    rast.set_timing(True)
    try:
        entry = search(lambda setting: rast.set_tuning(**setting),
                       lambda: _time(rast, prims, cameras, bg, dL, grads, images, reps), rast.tuning())
        rast.set_tuning(**entry["tuning"])
    finally:
        rast.set_timing(was_timing)
    store_cache(cache, key, entry)
    return entry
