"""Launch-geometry autotuner for views (``vgr_view_opts.grid_wide`` /
``grid_scan``), keyed by device, hierarchy and image size and cached in a
JSON file.

For a resolution class the tuner renders the same short walk with every
candidate geometry (each frame a captured CUDA graph, timed with CUDA events
on the view's stream after warm-up frames) and keeps the fastest.  Geometry
changes only how the work is spread over the 152 SMs, never the result, so
any cached choice is safe to reuse.
"""
from __future__ import annotations

import json
import os

from . import View

GRID_WIDE_PER_SM = (2, 4, 8, 16)   # grid-stride kernels: LoD, preprocess, colour, ranges
GRID_SCAN_PER_SM = (2, 3, 4, 6)    # ticketed look-back kernels: compaction, radix passes, emission


def cache_key(hier, width: int, height: int) -> str:
    import torch
    dev = torch.cuda.get_device_properties(torch.cuda.current_device())
    return "%s|sms=%d|nodes=%d|sh=%d|store=%d|%dx%d" % (dev.name, dev.multi_processor_count, hier.n_nodes,
                                                     hier.sh_degree, hier.storage, width, height)


def load_cache(path: str | None) -> dict:
    if path and os.path.exists(path):
        with open(path) as f:
            return json.load(f)
    return {}


def save_cache(path: str, cache: dict) -> None:
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _time_walk(hier, cams, tau, warmup: int, stream, **geom) -> float:
    import torch
    v = View(hier, use_graph=True, stream=stream.cuda_stream, **geom)
    try:
        for c in cams[:warmup]:
            v.render(c, tau)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for c in cams[warmup:]:
            v.render(c, tau)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / max(1, len(cams) - warmup)
    finally:
        v.close()


def tune(hier, cams, tau: float, *, cache_path: str | None = None, warmup: int = 3,
         wide=GRID_WIDE_PER_SM, scan=GRID_SCAN_PER_SM, force: bool = False) -> dict:
    """Best (grid_wide, grid_scan) for the image size of ``cams`` (all the
    same size): a cached entry unless ``force``; else every candidate is
    timed on the walk ``cams`` (the first ``warmup`` frames untimed).
    Returns {"grid_wide", "grid_scan", "ms", "default_ms", "candidates"}."""
    import torch
    W, H = int(cams[0]["width"]), int(cams[0]["height"])
    if not all(int(c["width"]) == W and int(c["height"]) == H for c in cams):
        raise ValueError("every camera of a tuning walk must have the same image size")
    key = cache_key(hier, W, H)
    cache = load_cache(cache_path)
    if key in cache and not force:
        return cache[key]
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    stream = torch.cuda.Stream()
    results = []
    for a in wide:
        for b in scan:
            ms = _time_walk(hier, cams, tau, warmup, stream, grid_wide=a * sms, grid_scan=b * sms)
            results.append((ms, a, b))
    results.sort()
    default = [ms for ms, a, b in results if a == 8 and b == 4]
    best_ms, a, b = results[0]
    entry = dict(grid_wide=a * sms, grid_scan=b * sms, ms=round(best_ms, 4),
                 default_ms=round(default[0], 4) if default else None,
                 candidates=[dict(wide_per_sm=x, scan_per_sm=y, ms=round(t, 4)) for t, x, y in results])
    if cache_path:
        cache = load_cache(cache_path)
        cache[key] = entry
        save_cache(cache_path, cache)
    return entry
