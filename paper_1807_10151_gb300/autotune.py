"""Tile-shape autotuner for the forward projector.

For a geometry it times supcg_project at every feasible rays-per-block tile
(32, 64, 96, 128) with CUDA events and keeps the fastest; results are cached
in a JSON file keyed by a geometry bucket (image size, views, bins, bin
spacing), so each bucket is measured once per cache file.  The tile does not
change results, only speed.
"""
from __future__ import annotations

import json
import os

CANDIDATES = (128, 96, 64, 32)
DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "tiling.json")


def bucket(G) -> str:
    return f"{G.nx}x{G.ny}_v{G.V}_u{G.U}_d{G.d:.6g}"


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def tune(G, reps=5, cache=DEFAULT_CACHE, force=False):
    """Choose and apply the fastest tile for G; returns {"tile": t, "ms": {...}}."""
    import torch
    db = _load(cache)
    key = bucket(G)
    if key in db and not force:
        G.set_tiling(db[key]["tile"])
        return db[key]
    x = torch.rand(G.ny, G.nx, device="cuda")
    y = torch.empty(G.V, G.U, device="cuda")
    st = torch.cuda.current_stream()
    times = {}
    for t in CANDIDATES:
        if G.set_tiling(t) != 0:
            continue
        G.project(x, out=y)                     # builds the workspace for this tiling
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(reps):
            G.project(x, out=y)
        e1.record(st)
        torch.cuda.synchronize()
        times[t] = e0.elapsed_time(e1) / reps
    best = min(times, key=times.get)
    G.set_tiling(best)
    rec = {"tile": best, "ms": {str(k): v for k, v in times.items()}}
    db[key] = rec
    os.makedirs(os.path.dirname(cache), exist_ok=True)
    with open(cache, "w") as f:
        json.dump(db, f, indent=1, sort_keys=True)
    return rec


BWD_CANDIDATES = (2, 3, 4, 5, 6, 8)


def tune_bwd(G, b, iters=4, reps=2, cache=DEFAULT_CACHE, force=False):
    """Choose and apply the backprojector's view parts per pixel tile for G by
    timing the backprojections of short profiled solves on data b (the solve's
    two-sinogram pass is what the setting serves); cached per geometry bucket.
    Unlike the forward tile, the setting changes the order of each pixel's sums
    (so the last bits of results).  Returns {"parts": p, "us": {...}}."""
    db = _load(cache)
    key = bucket(G) + "_bwd"
    if key in db and not force:
        G.set_bwd_parts(db[key]["parts"])
        return db[key]
    times = {}
    for p in BWD_CANDIDATES:
        if G.set_bwd_parts(p) != 0:
            continue
        G.solve_profiled(b, max_iter=1, graph=False)      # builds the workspace for this setting
        best = float("inf")
        for _ in range(reps):
            _, _, kinds = G.solve_profiled(b, max_iter=iters, graph=False)
            ms, n = kinds["backward"]
            best = min(best, ms / max(n, 1))
        times[p] = best * 1000.0
    best = min(times, key=times.get)
    G.set_bwd_parts(best)
    rec = {"parts": best, "us": {str(k): v for k, v in times.items()}}
    db[key] = rec
    os.makedirs(os.path.dirname(cache), exist_ok=True)
    with open(cache, "w") as f:
        json.dump(db, f, indent=1, sort_keys=True)
    return rec
