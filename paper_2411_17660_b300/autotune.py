"""Autotuner of the batched rasteriser's tile size and binning strategy.

The screen tile (8, 16 or 32 pixels) sets how many (Gaussian, tile) keys the
sort handles and how many warps share a tile's depth-sorted list; the binning
strategy ("tile": radix passes over the tile bits and a sort inside each
tile; "radix": radix passes over tile and depth bits) trades fewer global
passes against per-tile sorts that grow with the keys per tile.  Which pair
is fastest depends on the scene (Gaussian footprints) and the views.  The
tuner times one forward + backward per candidate on the caller's own inputs
(CUDA events on the current stream, after warm-up) and keeps the fastest,
cached per (GPU, N, SH degree, view sizes).  The images do not depend on
either choice, so it changes only speed.

The per-warp entry batch of the blend kernels is the warp width (32 entries
per chunk, one per lane) and is not a tuning parameter.
"""
from __future__ import annotations

import json
import os
from typing import Callable, Dict, Iterable, Optional, Sequence

TILES = (8, 16, 32)
BINNINGS = ("tile", "radix")
CANDIDATES = tuple(f"{t}/{b}" for t in TILES for b in BINNINGS)   # "tile size/binning"


def parse(candidate: str):
    """("16/tile") -> (16, "tile")."""
    t, b = candidate.split("/")
    return int(t), b


def signature(gpu: str, N: int, sh_degree: int, cams: Sequence) -> str:
    views = ",".join(f"{c.W}x{c.H}" for c in cams)
    return f"{gpu}|N={N}|deg={sh_degree}|views={views}"


def choose(time_ms: Callable[[object], float], candidates: Iterable = CANDIDATES) -> Dict[str, object]:
    """Times every candidate once with time_ms(candidate) and returns the
    fastest (ties go to the earlier candidate) with all timings."""
    times = {c: float(time_ms(c)) for c in candidates}
    best = min(times, key=lambda c: (times[c], list(times).index(c)))
    return {"best": best, "ms": times}


class TileCache:
    """Choices per signature, optionally persisted to a JSON file."""

    def __init__(self, path: Optional[str] = None):
        self.path = path
        self.entries: Dict[str, dict] = {}
        if path and os.path.exists(path):
            with open(path) as f:
                self.entries = json.load(f)

    def get(self, key: str) -> Optional[dict]:
        return self.entries.get(key)

    def put(self, key: str, value: dict):
        self.entries[key] = value
        if self.path:
            tmp = self.path + ".tmp"
            with open(tmp, "w") as f:
                json.dump(self.entries, f, indent=1, sort_keys=True)
            os.replace(tmp, self.path)


def tune(params, sh_degree: int, cams, viewmats, cache: Optional[TileCache] = None, reps: int = 3,
         warmup: int = 2, candidates: Iterable[str] = CANDIDATES) -> Dict[str, object]:
    """Times forward + backward (upstream gradient of ones on the colour) for
    each "tile size/binning" candidate on these inputs and returns
    {"tile": size, "binning": strategy, "ms": {candidate: ms}}."""
    import torch

    from . import render as R

    gpu = torch.cuda.get_device_name()
    key = signature(gpu, int(params["means"].shape[1]), sh_degree, cams)
    if cache is not None and cache.get(key) is not None:
        return cache.get(key)
    P = R.pixel_offsets(cams)[-1]
    d_color = torch.ones(3 * P, device=params["means"].device)
    grads = {k: torch.empty_like(v) for k, v in params.items()}
    d_pose = torch.empty(len(cams), 6, device=params["means"].device)

    def time_ms(candidate: str) -> float:
        tile, binning = parse(candidate)
        rast = R.GaussianRasterizer(tile, binning=binning)
        color, depth, alpha, ws = rast.render_forward(params, sh_degree, cams, viewmats)
        ws = rast.alloc_workspace(int(params["means"].shape[1]), cams, int(rast.info(ws).keys * 1.1) + 8192)

        def step():
            rast.forward_raw(params, sh_degree, cams, viewmats, ws, color, depth, alpha)
            rast.backward_raw(params, sh_degree, cams, viewmats, ws, d_color, None, None, grads, d_pose)

        for _ in range(warmup):
            step()
        start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        best = float("inf")
        for _ in range(reps):
            start.record()
            step()
            end.record()
            end.synchronize()
            best = min(best, start.elapsed_time(end))
        return best

    chosen = choose(time_ms, candidates)
    tile, binning = parse(chosen["best"])
    result = {"tile": tile, "binning": binning, "ms": chosen["ms"]}
    if cache is not None:
        cache.put(key, result)
    return result
