#!/usr/bin/env python
"""Benchmark of the batched differentiable Gaussian rasteriser.

Metric: fwd+bwd Mpix/s and mapping iterations/s of an 8-keyframe mapping
window (8 x 640x480 views, 100k Gaussians, SH degree 3; the renderer's
camera batch of the paper, Supp. Sec. 1.2), against the same window as 8
per-view launches.  One step = forward render of the window + L1 colour and
depth loss + backward to every Gaussian parameter and the 8 keyframe poses,
captured once as a CUDA graph and replayed (the eagerly launched step is
reported beside it).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gsr|reference]

Under torchrun (N > 1) every rank renders its own copy of the window (the
path does not shard here: replicas only); value = all pixels of all ranks /
max step time over ranks.  --impl reference times the FP64 CPU oracle on a
bounded crop of the same window (rank 0 only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fwd+bwd Mpix/s & mapping it/s (8-view batch) vs per-view launches; % FP32/SFU peak"
# Eq. "rnd_loss" weights of the paper's Replica setting (lambda1, lambda2)
PAPER_LAMBDA1, PAPER_LAMBDA2 = 0.8, 0.2
LOSS_NAMES = {"l1": "L1 colour/depth loss", "paper": "L1 + SSIM colour / L1 depth loss (0.8, 0.2)"}
FWD_OPS_PER_PAIR = 17   # FP32-pipe instructions per composited (pixel, Gaussian) pair, blend forward
STAGE_SLEEP_CYCLES = 4_000_000   # about 2 ms of GPU sleep before each stage-timing step
BWD_OPS_PER_PAIR = 48   # the same for the blend backward (before the per-warp reduction)
SURFEL_FWD_OPS_PER_PAIR = 47   # surfels: ray-disk intersection + compositing with normal and distortion
SURFEL_BWD_OPS_PER_PAIR = 85   # surfels: recomputed intersection + its backward
# MUFU (SFU) operations per composited pair: ex2 of alpha in the forward; ex2 and the
# reciprocal of 1 - alpha in the backward
MUFU_PER_PAIR = {"blend_fwd": 1, "blend_bwd": 2}
MUFU_PER_SM_CLK = 16   # SFU lanes per SM per clock (4 per SM sub-partition)
# peak device allocation allowed for the in-the-wild window (32 x 1920x1080, 2M Gaussians)
HBM_BUDGET_BYTES = {"outdoor": 32 * 10**9}
L2_FLUSH_BYTES = 256 << 20


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="gsr", choices=["gsr", "reference"])
    p.add_argument("--tile", type=int, default=16)
    p.add_argument("--workload", default="window", choices=["small", "room", "window", "uneven", "outdoor"],
                   help="window (8 x 640x480, 100k Gaussians) is the metric's workload; the others are for reports")
    p.add_argument("--loss", default="l1", choices=["l1", "paper"],
                   help="l1: L1 colour + weighted L1 depth; paper: the mixed L1 + SSIM + depth loss (0.8, 0.2)")
    p.add_argument("--separate-loss", action="store_true",
                   help="run the L1 loss as its own kernel after the forward (gsr_render + gsr_l1_loss) instead of "
                        "fused into the forward blend (gsr_render_l1)")
    p.add_argument("--primitive", default="gaussians", choices=["gaussians", "surfels"],
                   help="surfels: the 2-D surfel renderer (with normal and distortion outputs and gradients)")
    p.add_argument("--median", action="store_true", help="also render median depth and feed it a gradient")
    p.add_argument("--densify", action="store_true", help="also gather densification statistics in the backward")
    p.add_argument("--density-ops", action="store_true",
                   help="also time the density-control calls (ADC, MCMC relocation and noise) at 2M Gaussians")
    p.add_argument("--binning", default="tile", choices=["tile", "radix"],
                   help="tile binning strategy: per-tile counting sort (default) or onesweep radix sort")
    p.add_argument("--autotune", action="store_true",
                   help="pick the tile size, binning and entry batch with the autotuner first")
    p.add_argument("--batch", type=int, default=32, choices=[32, 64],
                   help="list entries a blend warp stages per round")
    p.add_argument("--fwd-rows", type=int, default=0, choices=[0, 8, 16],
                   help="pixel rows of a forward blend warp's block (0: the library's default, 16)")
    p.add_argument("--no-graph", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-per-view", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=12.0, help="target length of the CPU baseline sample")
    p.add_argument("--extra-workloads", default="uneven,outdoor",
                   help="comma-separated workloads also measured after the headline one (rank 0 of a 1-GPU run, "
                        "graph replay, autotuned tile, binning and batch), or 'none'")
    return p.parse_args()


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return dict(hbm_gbs=d["hbm_gbs"], sm_max_mhz=d.get("sm_max_mhz", 2032.0), source="measured")
    return dict(hbm_gbs=6400.0, sm_max_mhz=2032.0, source="fallback")


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.out, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.out.close()
        sm, mx, reasons = [], [], set()
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for name, val in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"),
                                     parts[5:9]):
                    if val.lower() == "active":
                        reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


# ------------------------------------------------------------------ distributed
def dist_setup(args=None):
    """Joins the torchrun process group (one rank per GPU, NCCL; gloo on a
    host without GPUs, where only the host-side logic runs)."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        import torch
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
            dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        else:
            dist.init_process_group("gloo")
    return ws, rank, local


def dist_barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def dist_max(ws, x: float) -> float:
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------ workload
def make_scene(name="window"):
    from paper_2411_17660_b300 import scenes
    return scenes.make(name)


def resolution(scene):
    sizes = sorted({f"{c.W}x{c.H}" for c in scene.cameras})
    return sizes[0] if len(sizes) == 1 else "mixed:" + ",".join(sizes)


def crop_pixels(scene, w, h):
    pix = []
    for c in scene.cameras:
        cw, ch = min(w, c.W), min(h, c.H)
        x0, y0 = (c.W - cw) // 2, (c.H - ch) // 2
        ys, xs = np.mgrid[y0:y0 + ch, x0:x0 + cw]
        pix.append((ys * c.W + xs).reshape(-1).astype(np.int64))
    return pix


def oracle_step(scene, pix, gC, gD):
    import oracle
    gA = [np.zeros(len(p)) for p in pix]
    return oracle.render_backward(scene, gC, gD, gA, pixels=pix)[0]


def oracle_sample(scene, seconds):
    """Picks a centred crop per view whose oracle fwd+bwd takes ~seconds."""
    import oracle
    oracle.build()
    rng = np.random.default_rng(0)

    def run(w, h):
        pix = crop_pixels(scene, w, h)
        gC = [rng.uniform(-1, 1, (3, len(p))) for p in pix]
        gD = [rng.uniform(-0.1, 0.1, len(p)) for p in pix]
        t0 = time.perf_counter()
        res = oracle_step(scene, pix, gC, gD)
        return time.perf_counter() - t0, pix, gC, gD, res

    w, h = 32, 24
    t = run(w, h)[0]
    t0 = run(2, 2)[0]                       # projection + binning cost, no pixels
    per_px = max(t - t0, 1e-9) / (w * h * scene.V)
    target_px = max((seconds - t0) / per_px / scene.V, 64)
    side = int(np.sqrt(target_px * 4 / 3))
    w = int(min(scene.cameras[0].W, max(8, side)))
    h = int(min(scene.cameras[0].H, max(6, side * 3 // 4)))
    return w, h, run


def cpu_baseline(scene, seconds, images=None):
    """The oracle's fwd+bwd on a crop; with images (per view (colour [3, H W],
    depth [H W]) of the timed GPU steps) also the parity of those pixels."""
    w, h, run = oracle_sample(scene, seconds)
    t, pix, _, _, res = run(w, h)
    npx = sum(len(p) for p in pix)
    out = {"value": npx / t / 1e6, "unit": "Mpix/s", "cores": os.cpu_count(), "kind": "oracle",
           "sample": f"fwd+bwd of a centred {w}x{h} crop (or less) of each of the {scene.V} views "
                     f"({npx} px, all {scene.N} Gaussians projected), {t:.1f} s, FP64"}
    if images is not None:
        worst_c = worst_d = all_c = all_d = 0.0
        near = over = 0
        for (col, dep), p, r in zip(images, pix, res):
            # pixels away from every FP32-vs-FP64 decision flip: threshold decisions (cutoff, alpha
            # skip, stop) farther than 1e-5 relative, depth order farther than 1e-6
            ok = (r["margin"] >= 1e-5) & (r["zmargin"] >= 1e-6)
            near += int((~ok).sum())
            dc = np.abs(col[:, p] - r["color"]).max(axis=0)
            dd = np.abs(dep[p] - r["depth"]) / np.maximum(np.abs(r["depth"]), 1e-3)
            worst_c = max(worst_c, float(dc[ok].max(initial=0.0)))
            worst_d = max(worst_d, float(dd[ok].max(initial=0.0)))
            all_c = max(all_c, float(dc.max(initial=0.0)))
            all_d = max(all_d, float(dd.max(initial=0.0)))
            over += int(((dc > 1e-4) | (dd > 1e-4)).sum())
        out["parity"] = {"pixels": npx, "near_threshold_pixels": near, "near_threshold_share": near / max(npx, 1),
                         "max_abs_color": worst_c,
                         "max_rel_depth": worst_d, "max_abs_color_all_pixels": all_c,
                         "max_rel_depth_all_pixels": all_d, "pixels_over_tolerance": over,
                         "tolerance": {"color": 1e-4, "depth": 1e-4},
                         "within": worst_c <= 1e-4 and worst_d <= 1e-4}
    return out


def reference_arm(args, ws, rank):
    if rank != 0:
        return
    scene = make_scene(args.workload)
    per_step = max(2.0, min(6.0, 120.0 / max(args.steps + args.warmup, 1)))
    w, h, run = oracle_sample(scene, per_step)
    for _ in range(args.warmup):
        run(w, h)
    times = []
    npx = 0
    for _ in range(args.steps):
        t, pix = run(w, h)[:2]
        times.append(t)
        npx = sum(len(p) for p in pix)
    ms = 1000 * statistics.mean(times)
    value = npx / (ms / 1000) / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Mpix/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": scene.name, "views": scene.V, "resolution": resolution(scene), "gaussians": scene.N,
                   "sh_degree": scene.sh_degree, "sample": f"{w}x{h} centred crop per view"},
        "cpu_baseline": {"value": value, "unit": "Mpix/s", "cores": os.cpu_count(), "kind": "oracle",
                         "sample": f"fwd+bwd of a centred {w}x{h} crop of each view, per step"},
        "e2e": {"value": value, "unit": "Mpix/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


class Window:
    """Device state of one mapping window (inputs, outputs, workspace)."""

    def __init__(self, scene, rast, views=None, dev="cuda", loss="l1", primitive="gaussians", median=False,
                 densify=False, fuse_l1=True):
        import torch
        from paper_2411_17660_b300 import render as R
        self.R, self.torch = R, torch
        idx = list(range(scene.V)) if views is None else views
        self.scene = scene
        self.loss_kind = loss
        self.fuse_l1 = fuse_l1 and loss == "l1" and primitive == "gaussians"
        self.surfels = primitive == "surfels"
        self.median, self.densify = median, densify
        self.cams = [R.Intrinsics(scene.cameras[v].H, scene.cameras[v].W, scene.cameras[v].fx,
                                  scene.cameras[v].fy, scene.cameras[v].cx, scene.cameras[v].cy) for v in idx]
        self.params = {k: torch.from_numpy(np.ascontiguousarray(getattr(scene, k), np.float32)).to(dev)
                       for k in R.PARAM_NAMES}
        self.vm = torch.from_numpy(np.stack([scene.cameras[v].T_cw for v in idx]).astype(np.float32)).to(dev)
        self.tc = torch.from_numpy(np.concatenate([scene.target_color[v].reshape(-1) for v in idx])).to(dev)
        self.td = torch.from_numpy(np.concatenate([scene.target_depth[v].reshape(-1) for v in idx])).to(dev)
        self.P = sum(c.H * c.W for c in self.cams)
        self.rast = rast
        self.color = torch.empty(3 * self.P, device=dev)
        self.depth = torch.empty(self.P, device=dev)
        self.alpha = torch.empty(self.P, device=dev)
        self.dC = torch.empty_like(self.color)
        self.dD = torch.empty_like(self.depth)
        self.loss = torch.empty(1, device=dev)
        self.grads = {k: torch.empty_like(v) for k, v in self.params.items()}
        self.d_pose = torch.empty(len(self.cams), 6, device=dev)
        # extra outputs and their (fixed) upstream gradients
        self.med = torch.empty(self.P, device=dev) if median else None
        self.dM = torch.full((self.P,), 1e-3, device=dev) if median else None
        self.normal = torch.empty(3 * self.P, device=dev) if self.surfels else None
        self.dist = torch.empty(self.P, device=dev) if self.surfels else None
        self.dN = torch.full((3 * self.P,), 1e-3, device=dev) if self.surfels else None
        self.dL = torch.full((self.P,), 1e-3, device=dev) if self.surfels else None
        self.dens = {k: torch.empty(scene.N, device=dev) for k in ("grad", "count", "radius")} if densify else None
        _, _, _, self.ws = rast.render_forward(self.params, scene.sh_degree, self.cams, self.vm)
        info = rast.info(self.ws)
        keys = info.keys
        if self.surfels:   # the surfels' tile bounds give their own key count
            cap = int(keys * 2) + 8192
            for _ in range(6):
                self.ws = rast.alloc_workspace(scene.N, self.cams, cap, dev)
                rast.surfels_forward_raw(self.params, scene.sh_degree, self.cams, self.vm, self.ws, self.color)
                info = rast.info(self.ws)
                if info.status == 0:
                    break
                cap = int(info.keys * 1.25) + 8192
            keys = info.keys
        # headroom so that the timed steps never re-grow
        self.ws = rast.alloc_workspace(scene.N, self.cams, int(keys * 1.1) + 8192, dev)

    def step(self, accumulate=False):
        R, sc = self.R, self.scene
        if self.surfels:
            self.rast.surfels_forward_raw(self.params, sc.sh_degree, self.cams, self.vm, self.ws, self.color,
                                          self.depth, self.alpha, self.normal, self.dist)
        elif self.fuse_l1:   # the forward blend also takes the L1 loss
            self.rast.forward_l1_raw(self.params, sc.sh_degree, self.cams, self.vm, self.ws, self.color, self.depth,
                                     self.alpha, self.tc, self.td, 1.0, sc.depth_weight, self.dC, self.dD, self.loss,
                                     self.med)
        else:
            self.rast.forward_raw(self.params, sc.sh_degree, self.cams, self.vm, self.ws, self.color, self.depth,
                                  self.alpha, self.med)
        if self.fuse_l1:
            pass
        elif self.loss_kind == "l1":
            R.l1_loss(self.rast, self.cams, self.vm, self.color, self.depth, self.tc, self.td, 1.0,
                      sc.depth_weight, self.dC, self.dD, self.loss)
        else:
            R.rgbd_loss(self.rast, self.cams, self.vm, self.color, self.depth, self.tc, self.td, PAPER_LAMBDA1,
                        PAPER_LAMBDA2, self.dC, self.dD, self.loss)
        if self.surfels:
            self.rast.surfels_backward_raw(self.params, sc.sh_degree, self.cams, self.vm, self.ws, self.dC, self.dD,
                                           None, self.dN, self.dL, self.grads, self.d_pose, accumulate=accumulate)
        else:
            self.rast.backward_raw(self.params, sc.sh_degree, self.cams, self.vm, self.ws, self.dC, self.dD, None,
                                   self.grads, self.d_pose, accumulate=accumulate, d_median_depth=self.dM,
                                   densify=self.dens)


def stage_rooflines(stage_ms, ops, pairs, alu_peak, hbm_gbs, scene, P, keys, binning="tile", tiles=1, sfu_peak=None,
                    visible=0):
    """Every stage against its bound: the blends against the FP32 lanes
    (composited pairs x FP32 instructions per pair) and, beside it, the SFU
    (composited pairs x MUFU operations per pair), the rest against HBM with
    their algorithmic bytes: what the stage must read and write once, from
    the Gaussian, pair, visible-pair (counted on the device) and key counts."""
    K = (scene.sh_degree + 1) ** 2
    param_b = scene.N * 4 * (3 + 3 + 4 + 1 + 3 * K)
    VN = scene.V * scene.N
    out = {}
    for s in ("blend_fwd", "blend_bwd"):
        a = pairs * ops[s] / (stage_ms[s] * 1e-3) / 1e9
        out[s] = {"bound": "alu", "achieved": a, "peak": alu_peak, "unit": "Gop/s", "frac": a / alu_peak}
        if sfu_peak and s in MUFU_PER_PAIR and stage_ms[s] > 0:
            m = pairs * MUFU_PER_PAIR[s] / (stage_ms[s] * 1e-3) / 1e9
            out[s]["sfu"] = {"achieved": m, "peak": sfu_peak, "unit": "Gop/s", "frac": m / sfu_peak,
                             "work": f"{MUFU_PER_PAIR[s]} MUFU per composited pair"}
    hbm = {
        # parameters once; per pair its tile count and densification radius; per visible pair its
        # 64-byte record; per emitted key its tile and word (per-tile binning).  The gradient rows are
        # cleared by the backward after use, not here.
        "preprocess": (param_b + 8 * VN + 64 * visible + (12 * keys if binning == "tile" else 0),
                       "parameters once + 8 B per pair + 64 B per visible pair (record)"
                       + (" + 12 B per key" if binning == "tile" else "")),
        # per-tile: count reads tile ids; scatter reads tile ids and words, writes words; tile sort
        # reads words, writes ids.  radix: 24 B per key per 8-bit pass (sort) + 8 (ranges)
        "sort": (36 * keys, "36 B per key") if binning == "tile" else
                (24 * keys * ((32 + max(1, (tiles - 1).bit_length()) + 7) // 8), "24 B per key per pass"),
        # parameters in, gradients out, a count per pair, each visible pair's gradient row read and
        # cleared and its stored colour read
        "preprocess_bwd": (2 * param_b + 4 * VN + 96 * visible,
                           "2 x parameters + 4 B per pair + 96 B per visible pair (gradient row read and cleared, "
                           "colour read)"),
    }
    if binning != "tile":
        # radix: counts read by the scan and the duplication, the record fields the spans use (centre,
        # factor, s_max, covariance, depth) read per visible pair, 12 B written per key
        hbm["scan_duplicate"] = (8 * VN + 52 * visible + 12 * keys,
                                 "8 B per pair + 52 B per visible pair + 12 B per key")
    for s, (b, note) in hbm.items():
        if s not in stage_ms or stage_ms[s] <= 0:
            continue
        a = b / (stage_ms[s] * 1e-3) / 1e9
        out[s] = {"bound": "hbm", "achieved": a, "peak": hbm_gbs, "unit": "GB/s", "frac": a / hbm_gbs,
                  "bytes": b, "note": note}
    return out


def launches_per_step(rast, win):
    info = rast.info(win.ws)
    tiles = info.tiles
    tbits = 1
    while (1 << tbits) < tiles:
        tbits += 1
    # init, preprocess, 3 scan kernels, duplicate, histogram, the radix
    # passes, ranges, blend, loss, blend backward, preprocess backward, pose
    # sums; per-tile binning emits its keys in the preprocess (no scan, no
    # duplicate), groups the keys by tile -- up to 32,768 tiles with a count (with
    # the scan in its last block) and a scatter, beyond with a histogram, the radix passes over the
    # tile bits and the ranges -- and adds 2 tile sorts; the L1 loss fused into
    # the forward blend has no kernel of its own
    loss = 0 if win.fuse_l1 else 1
    # beyond 32,768 tiles, and with radix binning, two kernels also list the
    # blends' tile order up to 65,536 tiles (the bucket count lists it
    # itself); not for surfels
    order = 0 if win.surfels or tiles > 65536 else 2
    group = 2 if tiles <= 32768 else 2 + (tbits + 7) // 8 + order
    if rast.binning == "tile" and not win.surfels:
        return 6 + loss + group + 2
    if rast.binning == "tile":   # surfels: scan + duplicate, then the same grouping
        return 10 + loss + group + 2
    return 12 + loss + (32 + tbits + 7) // 8 + order


def time_steps(torch, fn, K, flush, events_per_step=None):
    """Device time of K steps (CUDA events on the current stream), with an L2
    flush before each step outside the timed events."""
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    for k in range(K):
        flush()
        if events_per_step is not None:
            events_per_step(k)
        starts[k].record()
        fn()
        ends[k].record()
    torch.cuda.synchronize()
    return [s.elapsed_time(e) for s, e in zip(starts, ends)]


def traffic_for(kernel: str, workload: str):
    """DRAM bytes per launch from the committed ncu summary of this workload,
    if the kernel's source has not changed since the capture."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    name = "blend.cu" if "blend" in kernel else ("binning.cu" if kernel in ("sort", "duplicate") else "preprocess.cu")
    src = os.path.join(ROOT, "paper_2411_17660_b300", "csrc", name)
    kernel = "onesweep" if kernel == "sort" else kernel
    if not os.path.exists(path):
        return None
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    for line in open(path):
        if line.startswith("#"):
            continue
        f = dict(kv.split("=", 1) for kv in line.split() if "=" in kv)
        if f.get("kernel") == kernel and f.get("source_sha") == sha and f.get("workload") == workload:
            return float(f["dram_bytes_per_launch"])
    return None


def step_memory(torch, scene, win):
    """Peak device allocation of the step: every tensor of the window
    (parameters, targets, images, gradients, workspace) plus whatever the step
    allocates on the fly, read after the timed steps (the peak statistics
    were reset once the window was set up)."""
    peak = torch.cuda.max_memory_allocated() - L2_FLUSH_BYTES   # the flush buffer is alive throughout
    out = {"peak_allocated_bytes": int(peak), "workspace_bytes": int(win.ws.numel() * win.ws.element_size()),
           "note": "torch.cuda.max_memory_allocated() over the timed steps: parameters, targets, images, "
                   "gradients and the library's workspace (the library allocates nothing itself); "
                   "excludes the bench's 256 MB L2-flush buffer"}
    budget = HBM_BUDGET_BYTES.get(scene.name.split("-")[0])
    if budget:
        out["budget_bytes"] = budget
        out["within_budget"] = peak <= budget
    return out


def measure_workload(name, torch, B, R, flush, peaks, alu_peak, sfu_peak, K=5, W=3):
    """Another workload, measured like the headline one: tile size, binning
    and entry batch from the autotuner, stage times from eager steps queued behind a
    GPU sleep, the step as one replayed CUDA graph, the peak allocation."""
    from paper_2411_17660_b300 import autotune as A
    scene = make_scene(name)
    params = {k: torch.from_numpy(np.ascontiguousarray(getattr(scene, k), np.float32)).cuda() for k in R.PARAM_NAMES}
    cams = [R.Intrinsics(c.H, c.W, c.fx, c.fy, c.cx, c.cy) for c in scene.cameras]
    vm = torch.from_numpy(np.stack([c.T_cw for c in scene.cameras]).astype(np.float32)).cuda()
    tuned = A.tune(params, scene.sh_degree, cams, vm)
    del params, vm
    torch.cuda.empty_cache()
    rast = R.GaussianRasterizer(tuned["tile"], binning=tuned["binning"], batch=tuned["batch"],
                                fwd_rows=tuned["fwd_rows"])
    win = Window(scene, rast)
    torch.cuda.synchronize()
    torch.cuda.reset_peak_memory_stats()
    for _ in range(W):
        flush()
        win.step()
    ev_sets = [[torch.cuda.Event(enable_timing=True) for _ in range(B.STAGE_EVENTS)] for _ in range(K)]
    for es in ev_sets:    # stages a path skips keep these recordings (zero length)
        for e in es:
            e.record()
    torch.cuda.synchronize()
    for k in range(K):
        flush()
        torch.cuda._sleep(STAGE_SLEEP_CYCLES)
        rast.ctx.set_stage_events([e.cuda_event for e in ev_sets[k]])
        win.step()
    torch.cuda.synchronize()
    rast.ctx.set_stage_events(None)
    eager = statistics.mean(time_steps(torch, win.step, K, flush))
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        win.step()
    for _ in range(3):
        flush()
        graph.replay()
    replay = statistics.mean(time_steps(torch, graph.replay, K, flush))
    info = rast.info(win.ws)
    if info.status != 0:
        raise RuntimeError(f"{name}: device status {B.STATUS.get(info.status)}")
    stage_ms = {}
    for k, st in enumerate(B.STAGES):
        a, b = B.STAGE_SPANS[k]
        stage_ms[st] = statistics.mean(ev_sets[i][a].elapsed_time(ev_sets[i][b]) for i in range(K))
    ops = {"blend_fwd": FWD_OPS_PER_PAIR, "blend_bwd": BWD_OPS_PER_PAIR}
    roof = stage_rooflines(stage_ms, ops, info.pairs_contributing, alu_peak, peaks["hbm_gbs"], scene, win.P,
                           info.keys, tuned["binning"], info.tiles, sfu_peak, info.pairs_visible)
    out = {"config": {"workload": scene.name, "views": scene.V, "resolution": resolution(scene),
                      "gaussians": scene.N, "sh_degree": scene.sh_degree, "tile": tuned["tile"],
                      "binning": tuned["binning"], "batch": tuned["batch"], "fwd_rows": tuned["fwd_rows"],
                      "autotune_ms": tuned["ms"],
                      "step": f"forward + L1 colour/depth loss + backward (params + {scene.V} poses)",
                      "launch": "one CUDA graph per step, replayed", "steps": K, "warmup": W},
           "value": win.P / (replay / 1000) / 1e6, "unit": "Mpix/s", "ms_per_step": replay,
           "mapping_it_per_s": 1000.0 / replay, "eager_ms_per_step": eager,
           "stages_ms": stage_ms, "keys": info.keys, "pairs_contributing": info.pairs_contributing,
           "pairs_visible": info.pairs_visible,
           "stage_rooflines": roof, "memory": step_memory(torch, scene, win)}
    del graph, win
    return out


def main():
    args = parse()
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        reference_arm(args, world, rank)
        return
    import torch
    from paper_2411_17660_b300 import binding as B
    from paper_2411_17660_b300 import build as Build
    from paper_2411_17660_b300 import render as R
    Build.build()
    torch.cuda.set_device(local)
    scene = make_scene(args.workload)
    tile, tuned = args.tile, None
    if args.autotune:
        from paper_2411_17660_b300 import autotune as A
        w0 = Window(scene, R.GaussianRasterizer(16, binning=args.binning), loss=args.loss, primitive=args.primitive)
        tuned = A.tune(w0.params, scene.sh_degree, w0.cams, w0.vm)
        tile, args.binning, args.batch = tuned["tile"], tuned["binning"], tuned["batch"]
        args.fwd_rows = tuned["fwd_rows"]
        del w0
    rast = R.GaussianRasterizer(tile, binning=args.binning, batch=args.batch, fwd_rows=args.fwd_rows)
    opts = dict(loss=args.loss, primitive=args.primitive, median=args.median, densify=args.densify,
                fuse_l1=not args.separate_loss)
    flush_buf = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    flush = lambda: flush_buf.fill_(1.0)
    win = Window(scene, rast, **opts)
    torch.cuda.synchronize()
    torch.cuda.reset_peak_memory_stats()
    K, W = args.steps, args.warmup

    for _ in range(max(W, 3)):
        flush()
        win.step()
    torch.cuda.synchronize()

    # per-step stage events for the roofline (recorded inside the timed steps)
    ev_sets = [[torch.cuda.Event(enable_timing=True) for _ in range(B.STAGE_EVENTS)] for _ in range(K)]
    for s in ev_sets:
        for e in s:
            e.record()
    torch.cuda.synchronize()
    set_events = lambda k: rast.ctx.set_stage_events([e.cuda_event for e in ev_sets[k]])

    sampler = ClockSampler(local)
    dist_barrier(world)
    torch.cuda.synchronize()
    sampler.start()
    t0 = time.perf_counter()
    ms = time_steps(torch, win.step, K, flush, set_events)
    wall = time.perf_counter() - t0
    torch.cuda.synchronize()
    dist_barrier(world)
    rast.ctx.set_stage_events(None)
    ms_step = dist_max(world, statistics.mean(ms))

    # Per-stage device times (for the rooflines) from K more steps, each queued
    # behind a short GPU sleep so that the host has enqueued the whole step
    # before it runs: the eager steps above can be host-bound, and their stage
    # events then count the GPU's idle gaps too.
    rast.ctx.set_stage_events(None)
    for k in range(K):
        flush()
        torch.cuda._sleep(STAGE_SLEEP_CYCLES)
        set_events(k)
        win.step()
    torch.cuda.synchronize()
    rast.ctx.set_stage_events(None)

    info = rast.info(win.ws)
    if info.status != 0:
        raise RuntimeError(f"device status {B.STATUS.get(info.status)} during the timed steps")
    memory = step_memory(torch, scene, win)
    stage_ms = {}
    for k, name in enumerate(B.STAGES):
        a, b = B.STAGE_SPANS[k]
        stage_ms[name] = statistics.mean(ev_sets[i][a].elapsed_time(ev_sets[i][b]) for i in range(K))
    # the loss front end runs between the forward's last event and the backward's first
    stage_ms["loss"] = statistics.mean(ev_sets[i][5].elapsed_time(ev_sets[i][6]) for i in range(K))

    # the same window as 8 per-view launches
    per_view = None
    if not args.no_per_view:
        wins = [Window(scene, rast, [v], **opts) for v in range(scene.V)]

        def per_view_step():
            for i, w1 in enumerate(wins):
                w1.step(accumulate=i > 0)

        for _ in range(max(W, 3)):
            flush()
            per_view_step()
        pv = time_steps(torch, per_view_step, K, flush)
        per_view = dist_max(world, statistics.mean(pv))

    # the same step captured once in a CUDA graph and replayed
    graph_ms, graph = None, None
    if not args.no_graph:
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            win.step()
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            win.step()
        for _ in range(3):
            flush()
            graph.replay()
        gm = time_steps(torch, graph.replay, K, flush)
        graph_ms = dist_max(world, statistics.mean(gm))
    clocks = sampler.stop()   # sampled over every timed region above

    # end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        e2e = measure_e2e(torch, R, scene, win, K, W, flush)
        e2e["value"] = dist_max(world, -e2e["value"]) * -1 if world > 1 else e2e["value"]

    peaks = load_peaks()
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    alu_peak = n_sm * 128 * peaks["sm_max_mhz"] * 1e6 / 1e9   # Gop/s (FP32 lanes x clock)
    sfu_peak = n_sm * MUFU_PER_SM_CLK * peaks["sm_max_mhz"] * 1e6 / 1e9   # Gop/s (SFU lanes x clock)
    pairs = info.pairs_contributing
    dominant = max(("blend_fwd", "blend_bwd", "sort", "preprocess", "preprocess_bwd"), key=lambda s: stage_ms[s])
    ops = {"blend_fwd": FWD_OPS_PER_PAIR, "blend_bwd": BWD_OPS_PER_PAIR}
    if args.primitive == "surfels":
        ops = {"blend_fwd": SURFEL_FWD_OPS_PER_PAIR, "blend_bwd": SURFEL_BWD_OPS_PER_PAIR}
    if dominant in ops:
        achieved = pairs * ops[dominant] / (stage_ms[dominant] * 1e-3) / 1e9
        roof = {"kernel": dominant, "bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "Gop/s",
                "frac": achieved / alu_peak,
                "traffic": traffic_for(dominant, scene.name) if args.primitive == "gaussians" else None,
                "peak_note": f"FP32 lanes: {n_sm} SMs x 128 x {peaks['sm_max_mhz']:.0f} MHz (max clock)",
                "work": f"{pairs} composited pairs x {ops[dominant]} FP32 ops"}
    else:
        roof = {"kernel": dominant, "bound": "hbm", "achieved": None, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": None, "traffic": traffic_for(dominant, scene.name)}
    stage_roof = stage_rooflines(stage_ms, ops, pairs, alu_peak, peaks["hbm_gbs"], scene, win.P, info.keys,
                                 args.binning, info.tiles, sfu_peak if args.primitive == "gaussians" else None,
                                 info.pairs_visible)

    P_all = win.P * world
    # headline: the step as one replayed CUDA graph (the batched path's launch
    # mode); the eagerly launched step is reported beside it
    head_ms = graph_ms if graph_ms is not None else ms_step
    value = P_all / (head_ms / 1000) / 1e6
    line = {
        "metric": METRIC, "value": value, "unit": "Mpix/s", "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": head_ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": scene.name, "views": scene.V, "resolution": resolution(scene), "gaussians": scene.N,
                   "sh_degree": scene.sh_degree, "tile": tile, "binning": args.binning, "batch": args.batch,
                   "fwd_rows": rast.fwd_rows,
                   "autotune": tuned,
                   "step": f"forward + {LOSS_NAMES[args.loss]} + backward (params + {scene.V} poses)",
                   "loss_in_forward_blend": win.fuse_l1,
                   "primitive": args.primitive,
                   "extras": [k for k, on in (("median depth", args.median), ("densification statistics", args.densify),
                                              ("normal + distortion", args.primitive == "surfels")) if on],
                   "l2": "flushed before every step (256 MB write), outside the timed events",
                   "launch": "one CUDA graph per step, replayed" if graph_ms is not None else "eager launches",
                   "parallelism": "replicas" if world > 1 else "single"},
        "mapping_it_per_s": 1000.0 / head_ms,
        "eager": {"ms_per_step": ms_step, "value": P_all / (ms_step / 1000) / 1e6, "unit": "Mpix/s"},
        "per_view_launches": None if per_view is None else {
            "ms_per_step": per_view, "value": P_all / (per_view / 1000) / 1e6, "unit": "Mpix/s",
            "batched_speedup": per_view / ms_step, "note": "both launched eagerly"},
        "stages_ms": stage_ms,
        "stage_timing": "device time per stage from CUDA events, in steps queued behind a ~2 ms GPU sleep "
                        "so that host launch gaps do not count",
        "keys": info.keys, "pairs_contributing": pairs, "pairs_visible": info.pairs_visible,
        "memory": memory,
        "roofline": roof,
        "stage_rooflines": stage_roof,
        "graph_replay": None if graph_ms is None else {
            "ms_per_step": graph_ms, "value": P_all / (graph_ms / 1000) / 1e6, "unit": "Mpix/s"},
        "gpu_launches": launches_per_step(rast, win) * K,
        "clocks": clocks,
        "e2e": e2e,
        "wall_s": wall,
        "peaks_source": peaks["source"],
    }
    if args.density_ops:
        line["density_ops"] = measure_density(torch, win, K, W, flush, peaks["hbm_gbs"])

    if rank == 0 and not args.no_cpu:
        imgs = None
        if args.primitive == "gaussians":   # the oracle renders Gaussians
            cols = R.split_views(win.color, win.cams, 3)
            deps = R.split_views(win.depth, win.cams)
            imgs = [(c.reshape(3, -1).cpu().numpy().astype(np.float64), d.reshape(-1).cpu().numpy().astype(np.float64))
                    for c, d in zip(cols, deps)]
        line["cpu_baseline"] = cpu_baseline(scene, args.cpu_seconds, imgs)
    extras = [w for w in args.extra_workloads.split(",") if w and w != "none" and w != scene.name]
    if extras and world == 1 and args.primitive == "gaussians":
        del win, graph
        torch.cuda.empty_cache()
        line["workloads"] = {}
        for name in extras:
            line["workloads"][name] = measure_workload(name, torch, B, R, flush, peaks, alu_peak, sfu_peak,
                                                       K=min(K, 5), W=3)
            torch.cuda.empty_cache()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def measure_density(torch, win, K, W, flush, hbm_gbs, N_target=2_000_000):
    """Times the density-control calls on the workload's Gaussians tiled (and
    jittered) to 2M, the outdoor map size, with seeded statistics and draws.
    Roofline: algorithmic HBM bytes (parameters and statistics read once,
    outputs written once) over the measured time."""
    from paper_2411_17660_b300.density import DensityControl
    reps = max(1, N_target // win.scene.N)
    gen = torch.Generator(device="cuda").manual_seed(0)
    p = {k: (v.repeat(1, reps) if v.dim() == 2 else v.repeat(reps)).contiguous() for k, v in win.params.items()}
    N = int(p["means"].shape[1])
    p["means"] += 0.01 * torch.randn(p["means"].shape, device="cuda", generator=gen)
    deg = win.scene.sh_degree
    count = torch.randint(0, 9, (N,), device="cuda", generator=gen).float()
    grad = count * torch.empty(N, device="cuda").exponential_(1.0 / 2e-4, generator=gen)
    radius = 40.0 * torch.rand(N, device="cuda", generator=gen)
    normals = torch.randn((2, 3, N), device="cuda", generator=gen)
    draws = torch.randint(-(1 << 31), (1 << 31) - 1, (N,), device="cuda", dtype=torch.int32, generator=gen)
    eta = torch.randn((3, N), device="cuda", generator=gen)
    dc = DensityControl(win.rast)
    adc = dict(grad_threshold=2e-4, split_scale=0.02, min_opacity=0.005, max_screen_radius=30.0, max_world_scale=0.1)
    out, n_out = dc.densify_adc(p, deg, grad, count, radius, normals, sync=False, **adc)
    n_out = int(n_out.item())
    dead = int((torch.sigmoid(p["opacity_logits"]) <= 0.005).sum().item())
    noisy = torch.empty_like(p["means"])
    param_b = 4 * sum(v.shape[0] if v.dim() == 2 else 1 for v in p.values())   # bytes of one Gaussian
    ops = {
        "adc": (lambda: dc.densify_adc(p, deg, grad, count, radius, normals, sync=False, **adc),
                N * (param_b + 12) + n_out * param_b),
        "mcmc_relocate": (lambda: dc.mcmc_relocate(p, deg, draws, 0.005), N * (2 * param_b + 4)),
        "mcmc_noise": (lambda: dc.mcmc_noise(p, deg, eta, 1e4 * 1.6e-4, means_out=noisy), N * 68),
    }
    res = {"gaussians": N, "sh_degree": deg, "outputs_adc": n_out, "dead": dead,
           "note": "window Gaussians tiled to 2M; algorithmic bytes: parameters and statistics read once, "
                   "outputs written once; L2 flushed before each call"}
    for name, (fn, nbytes) in ops.items():
        for _ in range(max(W, 3)):
            fn()
        torch.cuda.synchronize()
        ms = statistics.mean(time_steps(torch, fn, K, flush))
        gbs = nbytes / (ms * 1e-3) / 1e9
        res[name] = {"ms": ms, "algorithmic_MB": nbytes / 1e6, "achieved_GBs": gbs, "frac_of_hbm": gbs / hbm_gbs}
    return res


def measure_e2e(torch, R, scene, win, K, W, flush):
    """Same step through the public API with pinned host inputs: H2D of the
    parameters, poses and targets, the step, D2H of the loss and pose grads.

    value: pipelined as a mapper would run it -- two sets of device inputs,
    the next step's inputs copied on a second stream while the current step
    computes (events order every copy after the last step that read its
    buffer, and every step after its own copies); one pair of events spans
    all K steps, so every step's copies and read-back are inside the timed
    region.  The step's data (parameters, targets, images, workspace) is
    larger than L2.  sequential: each step's copies, then the step, then the
    read-back, one step at a time with an L2 flush between steps (outside
    the timed events)."""
    names = list(R.PARAM_NAMES)
    host = {k: torch.from_numpy(np.ascontiguousarray(getattr(scene, k), np.float32)).pin_memory() for k in names}
    h_vm = torch.from_numpy(np.stack([c.T_cw for c in scene.cameras]).astype(np.float32)).pin_memory()
    h_tc = win.tc.cpu().pin_memory()
    h_td = win.td.cpu().pin_memory()
    out_loss = torch.empty(1, dtype=torch.float32).pin_memory()
    out_pose = torch.empty(scene.V, 6, dtype=torch.float32).pin_memory()
    h2d = sum(t.numel() * 4 for t in host.values()) + h_vm.numel() * 4 + h_tc.numel() * 4 + h_td.numel() * 4
    d2h = 4 + out_pose.numel() * 4
    out_grads = {k: torch.empty(v.shape, dtype=torch.float32).pin_memory() for k, v in win.grads.items()}
    d2h_all = d2h + sum(t.numel() * 4 for t in out_grads.values())

    def copy_in():
        for k in names:
            win.params[k].copy_(host[k], non_blocking=True)
        win.vm.copy_(h_vm, non_blocking=True)
        win.tc.copy_(h_tc, non_blocking=True)
        win.td.copy_(h_td, non_blocking=True)

    def read_back(grads):
        out_loss.copy_(win.loss, non_blocking=True)
        out_pose.copy_(win.d_pose, non_blocking=True)
        if grads:
            for k, t in out_grads.items():
                t.copy_(win.grads[k], non_blocking=True)

    # sequential
    def e2e_step(grads=False):
        copy_in()
        win.step()
        read_back(grads)

    for _ in range(max(W, 3)):
        flush()
        e2e_step()
    torch.cuda.synchronize()
    m_seq = statistics.mean(time_steps(torch, e2e_step, K, flush))

    # pipelined: buffer b holds the inputs of steps b, b + 2, ...
    bufs = [(win.params, win.vm, win.tc, win.td),
            ({k: torch.empty_like(v) for k, v in win.params.items()}, torch.empty_like(win.vm),
             torch.empty_like(win.tc), torch.empty_like(win.td))]
    main, side = torch.cuda.current_stream(), torch.cuda.Stream()
    copied = [torch.cuda.Event() for _ in range(2)]
    used = [torch.cuda.Event() for _ in range(2)]

    def use(b):
        win.params, win.vm, win.tc, win.td = bufs[b]

    def issue_copy(b):
        with torch.cuda.stream(side):
            side.wait_event(used[b])   # the last step that read buffer b has finished
            use(b)
            copy_in()
            copied[b].record(side)

    def run(steps, grads):
        issue_copy(0)
        for i in range(steps):
            b = i % 2
            if i + 1 < steps:
                issue_copy((i + 1) % 2)
            main.wait_event(copied[b])
            use(b)
            win.step()
            read_back(grads)
            used[b].record(main)

    def timed(grads):
        run(max(W, 3), grads)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(main)
        side.wait_event(e0)
        run(K, grads)
        e1.record(main)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / K

    m = timed(False)
    mg = timed(True)
    use(0)   # the window's own buffers again
    to = lambda ms: win.P / (ms / 1000) / 1e6
    return {"value": to(m), "unit": "Mpix/s", "ms_per_step": m,
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "pipelined": "the next step's inputs copied on a second stream while the current step computes; "
                         "one pair of events spans all steps, every step's copies and read-back included",
            "returns": "the loss and the pose gradients: the parameter gradients stay on the device, where the "
                       "mapper's optimiser consumes them",
            "with_param_grads": {"value": to(mg), "unit": "Mpix/s", "ms_per_step": mg,
                                 "d2h_bytes_per_step": d2h_all},
            "sequential": {"value": to(m_seq), "unit": "Mpix/s", "ms_per_step": m_seq,
                           "note": "copies, step and read-back one step at a time, L2 flushed between steps"}}


if __name__ == "__main__":
    main()
