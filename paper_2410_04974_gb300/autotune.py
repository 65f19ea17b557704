"""Autotuner for the render settings of a frame shape.

Times the complete forward + backward frame (every kernel of the library) on
the GPU for each candidate setting and keeps the fastest.  Candidates vary
the shared-memory batch, the persistent tile queue and, only when the caller
offers more than one, the tile shape.  Batch and persistence never change a
result; the tile shape does (the 3-sigma tile membership is part of the
render's definition), so the chosen shape is part of the returned settings
and must be the one any parity check uses.

Results are cached in a JSON file keyed by GPU name, scene size, SH degree,
camera sizes and the candidate space, so a frame shape is tuned once per
machine.
"""

from __future__ import annotations

import hashlib
import json
import os
import time

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "sixdgs", "autotune.json")


def candidate_space(tiles=((16, 16),), batches=(128, 256, 512, 1024), persistent=(False, True)):
    out = []
    for t in tiles:
        for b in batches:
            for p in persistent:
                out.append({"tile": [int(t[0]), int(t[1])], "batch": int(b), "persistent": bool(p)})
    return out


def signature(device_name, n, sh_degree, cams, space) -> str:
    sizes = [(int(c.width), int(c.height)) for c in cams]
    blob = json.dumps({"dev": device_name, "n": int(n), "deg": int(sh_degree), "sizes": sizes,
                       "space": space}, sort_keys=True)
    return hashlib.sha1(blob.encode()).hexdigest()


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(path, data):
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def measure_frame(params, n, sh_degree, cams, cand, steps=5, warmup=2, **render_kw):
    """Mean milliseconds of one forward + L1 + backward frame (the fused blend)
    with setting `cand`."""
    import torch

    from .render import Renderer

    r = Renderer(n, sh_degree, cams, tile=tuple(cand["tile"]), batch=cand["batch"],
                 persistent=cand["persistent"], **render_kw)
    img = r.forward(params)
    targets = torch.zeros_like(img)
    grads = r.new_grads(params)
    times = []
    for it in range(warmup + steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        r.condition_project(params)
        r.bin_sort()
        r.raster_fwd_bwd(img, targets)
        r.project_bwd(params, grads)
        e1.record()
        torch.cuda.synchronize()
        if it >= warmup:
            times.append(e0.elapsed_time(e1))
    r.raise_status()
    return sum(times) / len(times)


def tune(params, n, sh_degree, cams, space=None, cache=DEFAULT_CACHE, force=False, measure=None,
         device_name=None, **render_kw):
    """Fastest setting of `space` for this frame shape; returns
    {"tile", "batch", "persistent", "ms", "timings", "cached"}."""
    space = space or candidate_space()
    if device_name is None:
        import torch
        device_name = torch.cuda.get_device_name()
    key = signature(device_name, n, sh_degree, cams, space)
    data = _load(cache) if cache else {}
    if not force and key in data:
        hit = dict(data[key])
        hit["cached"] = True
        return hit
    measure = measure or (lambda c: measure_frame(params, n, sh_degree, cams, c, **render_kw))
    timings = []
    t0 = time.perf_counter()
    for cand in space:
        ms = float(measure(cand))
        timings.append(dict(cand, ms=ms))
    best = min(timings, key=lambda t: t["ms"])
    result = {"tile": best["tile"], "batch": best["batch"], "persistent": best["persistent"], "ms": best["ms"],
              "timings": timings, "seconds": round(time.perf_counter() - t0, 3)}
    if cache:
        data[key] = result
        _store(cache, data)
    result = dict(result)
    result["cached"] = False
    return result
