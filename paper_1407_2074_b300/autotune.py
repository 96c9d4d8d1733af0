"""Autotuner of the ray caster's launch shape.

For a given renderer and camera batch it times every candidate (warp tile shape x threads per
CTA x CTAs per SM) on a graph-captured render plan and keeps the fastest; the choice is cached per
(GPU name, workload key) in a JSON file ($VR_AUTOTUNE_CACHE, default ~/.cache/vr_b300/autotune.json).
"""
from __future__ import annotations

import json
import os

CANDIDATES = [
    (8, 4, 768, 1), (4, 8, 768, 1),
    (8, 4, 256, 8), (16, 2, 256, 8), (4, 8, 256, 8), (32, 1, 256, 8),
    (8, 4, 128, 16), (16, 2, 128, 16), (4, 8, 128, 16),
    (8, 4, 256, 2), (8, 4, 64, 32),
]


def cache_path():
    return os.environ.get("VR_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "vr_b300", "autotune.json"))


def _load():
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except Exception:
        return {}


def _store(d):
    p = cache_path()
    os.makedirs(os.path.dirname(p), exist_ok=True)
    tmp = p + ".tmp"
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
    os.replace(tmp, p)


def time_plan(plan, reps=5):
    import torch

    plan.launch()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        plan.launch()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def autotune(renderer, cams, key: str, mode=0, reps=5, use_cache=True, candidates=CANDIDATES):
    """Sets and returns the fastest launch shape (tile_w, tile_h, threads, ctas_per_sm) and the
    timings of all candidates (ms per batch)."""
    import torch

    full_key = f"{torch.cuda.get_device_name()}|{key}|mode{mode}"
    cache = _load() if use_cache else {}
    if full_key in cache:
        shape = tuple(cache[full_key]["shape"])
        renderer.set_launch_shape(*shape)
        return shape, cache[full_key].get("timings", {})
    timings = {}
    images = None
    for shape in candidates:
        renderer.set_launch_shape(*shape)
        plan = renderer.plan(cams, images, mode)
        images = plan.images
        timings["x".join(map(str, shape))] = time_plan(plan, reps)
        plan.close()
    best = min(timings, key=timings.get)
    shape = tuple(int(v) for v in best.split("x"))
    renderer.set_launch_shape(*shape)
    if use_cache:
        cache = _load()
        cache[full_key] = {"shape": list(shape), "timings": timings}
        _store(cache)
    return shape, timings
