"""Autotuner for the compositing configuration.

The compositor's tile shape and pixels per thread change only speed: every
supported configuration produces bit-identical images (each pixel's
arithmetic is the same expression; the tile binning is conservative for
the alpha gate).  So the tuner may pick any of them by time alone: it
renders the caller's workload (forward, optionally forward + backward) with
every candidate, times each with CUDA events, and returns the fastest.
Results are cached in a JSON file keyed by the workload's shape (Gaussian
count, SH degree, image sizes, whether the backward is included).
"""
from __future__ import annotations

import json
import os

import torch

from . import render as R

# every (tile width, tile height, pixels per thread) the library supports
CONFIGS = ((16, 16, 1), (16, 16, 2), (16, 16, 4), (8, 8, 1), (8, 8, 2), (16, 8, 1), (16, 8, 2), (32, 8, 1),
           (32, 16, 1), (32, 16, 2), (32, 16, 4), (32, 32, 4), (16, 32, 4))

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "pvg_gb300", "tune.json")


def workload_key(scene_t, cams, backward):
    n = int(scene_t["mu"].shape[0])
    deg = R.sh_degree(scene_t)
    sizes = ",".join("%dx%d" % (int(c["width"]), int(c["height"])) for c in cams)
    return "n=%d;deg=%d;views=%s;bwd=%d" % (n, deg, sizes, int(bool(backward)))


def _time_config(cfg, scene_t, cams, backward, warmup, iters):
    tw, th, px = cfg
    r = R.Renderer(tile=(tw, th), pixels_per_thread=px)
    fr = R.Frame()
    outs = r.alloc_images(cams)
    grads = {k: torch.empty_like(scene_t[k]) for k in R.PARAM_NAMES} if backward else None
    dls = [dict(rgb=torch.full_like(o["rgb"], 1e-3)) for o in outs] if backward else None

    def run():
        r.forward(scene_t, cams, outs=outs, frame=fr)
        if backward:
            r.backward(scene_t, cams, fr, dls, grads=grads)

    for _ in range(warmup):
        run()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record()
    for _ in range(iters):
        run()
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / iters
    fr.close()
    r.close()
    return ms


def tune(scene_t, cams, backward=True, warmup=2, iters=5, configs=CONFIGS, cache_path=None, use_cache=True):
    """Returns ((tile_w, tile_h, pixels_per_thread), {config: ms})."""
    key = workload_key(scene_t, cams, backward)
    path = cache_path or os.environ.get("PVG_TUNE_CACHE", DEFAULT_CACHE)
    cache = {}
    if use_cache and os.path.exists(path):
        try:
            with open(path) as f:
                cache = json.load(f)
        except (OSError, ValueError):
            cache = {}
        if key in cache:
            best = tuple(cache[key]["best"])
            return best, {tuple(json.loads(k)): v for k, v in cache[key]["table"].items()}
    table = {}
    for cfg in configs:
        table[tuple(cfg)] = _time_config(cfg, scene_t, cams, backward, warmup, iters)
    best = min(table, key=table.get)
    if use_cache:
        cache[key] = {"best": list(best), "table": {json.dumps(list(k)): v for k, v in table.items()}}
        try:
            os.makedirs(os.path.dirname(path), exist_ok=True)
            with open(path, "w") as f:
                json.dump(cache, f, indent=1)
        except OSError:
            pass
    return best, table
