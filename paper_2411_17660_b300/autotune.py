"""Autotuner of the batched rasteriser: tile size, binning strategy, the
blends' per-warp entry batch and the forward blend's block height.

The screen tile (8, 16 or 32 pixels) sets how many (Gaussian, tile) keys the
sort handles and how many warps share a tile's depth-sorted list; the binning
strategy ("tile": grouping by tile and a sort inside each tile; "radix":
radix passes over tile and depth bits) trades fewer global passes against
per-tile sorts that grow with the keys per tile; the batch (32 or 64 list
entries staged per warp and round in both blends) trades staging rounds and
loads in flight against entries staged past a warp's transmittance stop;
the forward blend's warp block of 8 columns by 16 or 8 rows trades entries
shared among more pixels against evaluations of entries that reach no pixel
of the block.  Which combination is fastest depends on the scene (Gaussian footprints) and
the views.  The timing runs in the library (gsr_autotune): forward +
backward per candidate on the caller's own inputs, CUDA events on the
stream, best of a few after a warm-up run.  This module sizes the workspace
for the candidate with the most keys and caches the choice per (GPU, N, SH
degree, view sizes) in an optional JSON file.  The images do not depend on
any of the choices, so tuning changes only speed.
"""
from __future__ import annotations

import json
import os
from typing import Dict, Optional, Sequence

TILES = (8, 16, 32)
BINNINGS = ("tile", "radix")
BATCHES = (32, 64)
FWD_ROWS = (16, 8)
# "tile size/binning/batch/forward rows", in the order the library times them (64 is not
# offered at tile 32, 16 rows not at tile 8)
CANDIDATES = tuple(f"{t}/{b}/{k}/{r}" for t in TILES for b in BINNINGS for k in BATCHES for r in FWD_ROWS
                   if not (t == 32 and k == 64) and not (t == 8 and r == 16))


def parse(candidate: str):
    """("16/tile/32/8") -> (16, "tile", 32, 8)."""
    t, b, k, r = candidate.split("/")
    return int(t), b, int(k), int(r)


def signature(gpu: str, N: int, sh_degree: int, cams: Sequence) -> str:
    views = ",".join(f"{c.W}x{c.H}" for c in cams)
    return f"{gpu}|N={N}|deg={sh_degree}|views={views}"


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


def tune(params, sh_degree: int, cams, viewmats, cache: Optional[TileCache] = None,
         reps: int = 3) -> Dict[str, object]:
    """Times every candidate with gsr_autotune on these inputs and returns
    {"tile": size, "binning": strategy, "batch": entries, "fwd_rows": rows,
    "ms": {candidate: ms or None when it could not run}}."""
    import torch

    from . import binding as B
    from . import render as R

    gpu = torch.cuda.get_device_name()
    N = int(params["means"].shape[1])
    key = signature(gpu, N, sh_degree, cams)
    if cache is not None and cache.get(key) is not None and "fwd_rows" in cache.get(key):
        return cache.get(key)
    dev = params["means"].device
    # a workspace with room for the keys of the smallest tile (the most keys)
    sizing = R.GaussianRasterizer(8)
    _, _, _, ws = sizing.render_forward(params, sh_degree, cams, viewmats)
    keys = sizing.info(ws).keys
    del ws
    rast = R.GaussianRasterizer(8)
    ws = rast.alloc_workspace(N, cams, int(keys * 1.1) + 8192, dev)
    P = R.pixel_offsets(cams)[-1]
    color, depth, alpha = (torch.empty(3 * P, device=dev), torch.empty(P, device=dev), torch.empty(P, device=dev))
    grads = {k: torch.empty_like(v) for k, v in params.items()}
    g = R.gaussians_struct(*[params[k] for k in R.PARAM_NAMES], sh_degree)
    views = R.view_structs(cams, viewmats, color, depth, alpha)
    out = B.Grads(*[grads[k].data_ptr() for k in R.PARAM_NAMES], 0, 0, 0, 0)
    st, entries = rast.ctx.autotune(g, views, out, ws.data_ptr(), ws.numel(), reps,
                                    torch.cuda.current_stream().cuda_stream)
    rast.ctx.check(st, "gsr_autotune")
    name = {B.BIN_TILE: "tile", B.BIN_RADIX: "radix"}
    times = {f"{e.tile}/{name[e.binning]}/{e.batch}/{e.fwd_rows}": (float(e.ms) if e.status == B.OK else None)
             for e in entries}
    ran = {c: t for c, t in times.items() if t is not None}
    best = min(ran, key=lambda c: (ran[c], list(times).index(c)))
    tile, binning, batch, rows = parse(best)
    result = {"tile": tile, "binning": binning, "batch": batch, "fwd_rows": rows, "ms": times}
    if cache is not None:
        cache.put(key, result)
    return result
