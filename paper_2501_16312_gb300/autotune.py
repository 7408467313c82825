"""Autotuner for the rasterizer's launch parameters.

The tuning knobs (sort mode, pixels per blend thread, records per shared-memory
batch, resident blend blocks per SM, one- or two-pass backward chain) change
only the schedule: every setting renders bit-identical images (the chain's
split only reorders the sum of a primitive's centre-gradient terms).  The
tuner times forward + backward of the caller's own workload with the
library's per-stage CUDA events, picks the sort mode by the sort stages, the
blend parameters by the two blend stages and the chain form by the chain
stage, and caches the choice as JSON keyed by GPU name, primitive kind and
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


def tune(rast, prims, cameras, bg=(0.0, 0.0, 0.0), dL=None, reps: int = 3,
         cache: Optional[str] = DEFAULT_CACHE, force: bool = False) -> dict:
    """Pick and apply the fastest tuning for this workload; returns it."""
    import torch
    gpu = torch.cuda.get_device_name(rast.device)
    key = cache_key(gpu, prims.kind, prims.n, cameras)
    if cache and not force and os.path.exists(cache):
        try:
            with open(cache) as f:
                known = json.load(f)
            if key in known:
                rast.set_tuning(**known[key]["tuning"])
                return known[key]
        except (OSError, ValueError):
            pass
    P = sum(c.width * c.height for c in cameras)
    images = torch.empty(3 * P, device=rast.device)
    if dL is None:
        dL = torch.ones(3 * P, device=rast.device)
    grads = dict(centre=torch.empty_like(prims.centre), verts=torch.empty_like(prims.verts),
                 opacity=torch.empty_like(prims.opacity), sh=torch.empty_like(prims.sh))
    was_timing = True
    rast.set_timing(True)
    base = rast.tuning()
    results = []
    # sort mode, judged on the sort stages at the current blend setting
    sort_times = {}
    for sm in (0, 1):
        rast.set_tuning(sort_mode=sm)
        t = _time(rast, prims, cameras, bg, dL, grads, images, reps)
        sort_times[sm] = sum(t[s] for s in SORT_STAGES)
        results.append({"sort_mode": sm, **t})
    best_sort = min(sort_times, key=sort_times.get)
    rast.set_tuning(sort_mode=best_sort)
    # blend schedule
    blend_times = {}
    for pix, batch, bps in itertools.product((2, 4), (32, 64), (0,)):
        rast.set_tuning(pixels_per_thread=pix, batch=batch, blocks_per_sm=bps)
        t = _time(rast, prims, cameras, bg, dL, grads, images, reps)
        blend_times[(pix, batch, bps)] = sum(t[s] for s in BLEND_STAGES)
        results.append({"pixels_per_thread": pix, "batch": batch, "blocks_per_sm": bps, **t})
    pix, batch, bps = min(blend_times, key=blend_times.get)
    rast.set_tuning(pixels_per_thread=pix, batch=batch, blocks_per_sm=bps)
    # the backward chain in one or two passes, judged on its own stage
    chain_times = {}
    for split in (0, 1):
        rast.set_tuning(chain_split=split)
        t = _time(rast, prims, cameras, bg, dL, grads, images, reps)
        chain_times[split] = t["chain"]
        results.append({"chain_split": split, **t})
    best_chain = min(chain_times, key=chain_times.get)
    rast.set_tuning(chain_split=best_chain)
    # when a backward warp reduces over its lanes rather than letting each
    # contributing lane add its own terms, judged on the backward blend
    sparse_times = {}
    for sl in (8, 16):
        rast.set_tuning(sparse_lanes=sl)
        t = _time(rast, prims, cameras, bg, dL, grads, images, reps)
        sparse_times[sl] = t["blend_bwd"]
        results.append({"sparse_lanes": sl, **t})
    best_sparse = min(sparse_times, key=sparse_times.get)
    choice = dict(base, sort_mode=best_sort, pixels_per_thread=pix, batch=batch, blocks_per_sm=bps,
                  chain_split=best_chain, sparse_lanes=best_sparse)
    rast.set_tuning(**choice)
    rast.set_timing(was_timing)
    entry = {"tuning": choice, "sort_ms": sort_times[best_sort],
             "blend_ms": blend_times[(pix, batch, bps)], "trials": results}
    if cache:
        try:
            os.makedirs(os.path.dirname(cache), exist_ok=True)
            known = {}
            if os.path.exists(cache):
                with open(cache) as f:
                    known = json.load(f)
            known[key] = entry
            with open(cache + ".tmp", "w") as f:
                json.dump(known, f, indent=1)
            os.replace(cache + ".tmp", cache)
        except (OSError, ValueError):
            pass
    return entry
