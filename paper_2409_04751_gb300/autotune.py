"""Autotuner for the rasterizers' work shape (pixels per thread, forward and backward).

Every shape renders the same image bit for bit (the per-pixel arithmetic does not depend on
it) and the same gradients up to the order of their floating-point sums, so the tuner is free
to pick whichever is fastest on the workload at hand.
It times each candidate with CUDA events on the caller's stream, after one untimed launch,
and caches the choice per (GPU, workload signature) in a small JSON file.
"""
import json
import os

import torch

from . import fgs

SHAPES = (1, 2, 4)
BWD_SHAPES = (1, 2, 4, 8)  # the backward also has a one-warp-per-tile shape
CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "tuning.json")


def _signature(frame, n):
    name = torch.cuda.get_device_name()
    tiles = frame.tile_ranges.numel() // 2
    return f"{name}|n={n}|tiles={tiles}|pix={frame.final_T.numel()}|views={len(frame.cams)}"


def _time(fn, reps):
    fn()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    start.record()
    for _ in range(reps):
        fn()
    end.record()
    end.synchronize()
    return start.elapsed_time(end) / reps


def tune_raster(renderer, gs, frame, dL_dimages, reps=3, use_cache=True):
    """Pick the fastest (forward, backward) pixels-per-thread for this frame's workload, set it
    as `renderer`'s work shape (renderer.set_shape; every later call of that renderer passes it
    in its fgs_options) and return {"fwd": ppt, "bwd": ppt, "ms": {...}}. Other renderers are
    not affected."""
    n = int(gs["means"].shape[0])
    sig = _signature(frame, n)
    cache = {}
    if use_cache and os.path.exists(CACHE):
        try:
            cache = json.load(open(CACHE))
        except (OSError, ValueError):
            cache = {}
    if use_cache and sig in cache:
        c = cache[sig]
        renderer.set_shape(c["fwd"], c["bwd"])
        return c
    ws = renderer._bufs["ws"]
    from .renderer import gaussians_of
    g = gaussians_of(gs)
    grads = {k: torch.empty_like(gs[k]) for k in ("means", "scales", "quats", "opacities", "sh")}
    ms = {}

    def fwd(f):
        fgs.fgs_rasterize(frame.records, frame.vals, frame.tile_ranges, frame.cams, frame.bg,
                          frame.images, frame.final_T, frame.n_processed, ws, ws.numel(),
                          opts=fgs.options(fwd=f))

    def bwd(b):
        fgs.fgs_backward_raster(frame.records, frame.vals, frame.tile_ranges, n, frame.cams,
                                frame.bg, frame.final_T, frame.n_processed, dL_dimages, ws,
                                ws.numel(), opts=fgs.options(bwd=b))

    for s in SHAPES:
        ms[f"fwd{s}"] = _time(lambda: fwd(s), reps)
    best_f = min(SHAPES, key=lambda s: ms[f"fwd{s}"])
    fwd(best_f)  # the backward reads the forward's per-pixel state
    for s in BWD_SHAPES:
        ms[f"bwd{s}"] = _time(lambda: bwd(s), reps)
    best_b = min(BWD_SHAPES, key=lambda s: ms[f"bwd{s}"])
    renderer.set_shape(best_f, best_b)
    # leave the frame's buffers as a plain forward + backward would
    fwd(best_f)
    bwd(best_b)
    fgs.fgs_backward_preprocess(g, frame.cams, frame.records, frame.tiles_touched,
                                grads["means"], grads["scales"], grads["quats"],
                                grads["opacities"], grads["sh"], ws, ws.numel())
    out = {"fwd": best_f, "bwd": best_b, "ms": ms}
    if use_cache:
        cache[sig] = out
        try:
            os.makedirs(os.path.dirname(CACHE), exist_ok=True)
            with open(CACHE, "w") as f:
                json.dump(cache, f, indent=1)
        except OSError:
            pass
    return out
