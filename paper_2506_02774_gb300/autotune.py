"""Autotuner for views: the launch geometry (``vgr_view_opts.grid_wide`` /
``grid_scan``), the tile size (``tile_size``: 8, 16 or 32 pixels) and the
blend's staging depth (``blend_depth``: Gaussians a warp stages per chunk),
keyed by device, hierarchy and image size and cached in a JSON file.

For a resolution class the tuner renders the same short walk with every
candidate geometry at the default tile and depth (each frame a captured CUDA
graph, timed with CUDA events on the view's stream after warm-up frames),
keeps the fastest, then tries every (tile, depth) at that geometry.  None of
the knobs changes the cut or the image (binning is exact at any tile size),
only how the work is cut up and spread over the SMs, so any cached choice is
safe to reuse.  ``tune_batch`` picks, on the batch itself, how many of a
batch's views run at once and the (tile, depth) of its single blend launch.
"""
from __future__ import annotations

import json
import os

from . import View

GRID_WIDE_PER_SM = (2, 4, 8, 16)   # grid-stride kernels: LoD, preprocess (with colour), ranges
GRID_SCAN_PER_SM = (2, 3, 4, 6)    # ticketed look-back kernels: compaction, radix passes, emission
BLEND_DEPTHS = (16, 32, 48)        # Gaussians a blend warp stages per chunk
BATCH_CHAINS = (0, 1, 2, 3, 4, 8)  # views of a batch running at once (0: all)
TILE_SIZES = (8, 16, 32)           # tile side in pixels


def _pairs(tiles, depths):
    """(tile, depth) candidates; 48-deep staging needs tiles of 16 or 32."""
    return [(t, d) for t in tiles for d in depths if not (t == 8 and d == 48)]


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
         wide=GRID_WIDE_PER_SM, scan=GRID_SCAN_PER_SM, depths=BLEND_DEPTHS, tiles=TILE_SIZES,
         force: bool = False) -> dict:
    """Best (grid_wide, grid_scan, tile_size, blend_depth) for the image size
    of ``cams`` (all the same size): a cached entry unless ``force``; else
    every geometry is timed on the walk ``cams`` (the first ``warmup`` frames
    untimed) with 16-pixel tiles and depth 32, then every (tile, depth) at the
    best geometry.
    Returns {"grid_wide", "grid_scan", "tile_size", "blend_depth", "ms", "default_ms", "candidates"}."""
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
            ms = _time_walk(hier, cams, tau, warmup, stream, grid_wide=a * sms, grid_scan=b * sms, tile_size=16,
                            blend_depth=32)
            results.append((ms, a, b, 16, 32))
    results.sort()
    default = [r[0] for r in results if r[1] == 8 and r[2] == 4]
    _, a, b, _, _ = results[0]
    for t, d in _pairs(tiles, depths):
        if (t, d) != (16, 32):
            ms = _time_walk(hier, cams, tau, warmup, stream, grid_wide=a * sms, grid_scan=b * sms, tile_size=t,
                            blend_depth=d)
            results.append((ms, a, b, t, d))
    results.sort()
    best_ms, a, b, t, d = results[0]
    entry = dict(grid_wide=a * sms, grid_scan=b * sms, tile_size=t, blend_depth=d, ms=round(best_ms, 4),
                 default_ms=round(default[0], 4) if default else None,
                 candidates=[dict(wide_per_sm=x, scan_per_sm=y, tile_size=z, blend_depth=q, ms=round(ms_, 4))
                             for ms_, x, y, z, q in results])
    if cache_path:
        cache = load_cache(cache_path)
        cache[key] = entry
        save_cache(cache_path, cache)
    return entry


def tune_batch(views, steps, taus, *, depths=BLEND_DEPTHS, tiles=TILE_SIZES, chains=BATCH_CHAINS,
               warmup: int = 2) -> dict:
    """The concurrency, tile size and staging depth of a batch
    (``vgr_render_batch`` runs the views' frames in parallel chains, then the
    blend of every view it can in one launch, at one tile size and depth):
    every number of chains is timed at 16-pixel tiles and depth 32, then every
    (tile, depth) at the best number, each set on all views and timed on the
    batch walk ``steps`` (a list of per-step camera lists; the first
    ``warmup`` steps untimed), wall clock per batch.  The fastest is left set.
    Returns {"chains", "tile_size", "blend_depth", "ms_per_batch", "candidates"}."""
    import time

    import torch

    from . import render_batch, set_batch_chains

    def run(c, t, d):
        set_batch_chains(c)
        for v in views:
            v.set_tuning(blend_depth=d, tile_size=t)
            v.reset()
        for cams in steps[:warmup]:
            render_batch(views, cams, taus)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for cams in steps[warmup:]:
            render_batch(views, cams, taus)
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) * 1e3 / max(1, len(steps) - warmup), c, t, d

    n = len(views)
    seen, results = set(), []
    for c in chains:
        eff = n if c == 0 else min(n, c)  # chains beyond the view count run like 0
        if eff not in seen:
            seen.add(eff)
            results.append(run(c, 16, 32))
    results.sort()
    c = results[0][1]
    for t, d in _pairs(tiles, depths):
        if (t, d) != (16, 32):
            results.append(run(c, t, d))
    results.sort()
    best_ms, c, t, d = results[0]
    set_batch_chains(c)
    for v in views:
        v.set_tuning(blend_depth=d, tile_size=t)
        v.reset()
    return dict(chains=c, tile_size=t, blend_depth=d, ms_per_batch=round(best_ms, 3),
                candidates=[dict(chains=x, tile_size=z, blend_depth=q, ms_per_batch=round(ms_, 3))
                            for ms_, x, z, q in results])
