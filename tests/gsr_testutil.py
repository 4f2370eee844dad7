"""Helpers shared by the GPU parity tests: move a seeded scene to the device,
run the CUDA path through the C ABI, and compare it with the FP64 oracle
under the tolerances of the specification:
  colour   |dC| <= 1e-4 absolute per channel
  depth    |dD| <= 1e-4 * max(|D_ref|, 1e-3)
  opacity  |dA| <= 1e-4 absolute
  gradients: relative L2 <= 1e-3 per parameter tensor.
Pixels where the oracle took a decision close to its threshold may be
FP32-vs-FP64 decision flips: those whose threshold margin (the relative
distance of a cutoff, alpha-skip or stop decision from its threshold) is
below MARGIN, or whose depth-order margin (the relative gap between two
consecutive depths) is below ZMARGIN.  Out-of-tolerance pixels among them
are counted, and their share must stay below FLIP_SHARE; every other pixel
must meet the tolerance.

MARGIN: the FP32 path computes d^2 from double-float pixel offsets and the
Cholesky factor of the inverse covariance, each a few ulps off, so d^2,
alpha = sigma exp(-d^2 / 2) and the transmittance product carry relative
errors of a few 1e-7 to 1e-6; 1e-5 leaves a factor of ten.
ZMARGIN: depths are sorted as FP32 values (the camera-frame z, formed with
a compensated dot product: half an ulp, 6e-8 relative), so two depths more
than one ulp (1.2e-7 relative) apart cannot swap; 1e-6 leaves a factor of
eight.
"""
from __future__ import annotations

import numpy as np
import torch

import oracle
from paper_2411_17660_b300 import render as R
from paper_2411_17660_b300.scenes import Scene

COLOR_TOL = 1e-4
DEPTH_TOL = 1e-4
ALPHA_TOL = 1e-4
GRAD_TOL = 1e-3
MARGIN = 1e-5
ZMARGIN = 1e-6
FLIP_SHARE = 1e-3
SURFEL_MARGIN = 1e-4     # the surfel oracle's single margin (ray-splat decisions)


def to_device(scene: Scene, dev="cuda"):
    params = {k: torch.from_numpy(np.ascontiguousarray(getattr(scene, k), dtype=np.float32)).to(dev)
              for k in R.PARAM_NAMES}
    cams = [R.Intrinsics(c.H, c.W, float(c.fx), float(c.fy), float(c.cx), float(c.cy)) for c in scene.cameras]
    viewmats = torch.from_numpy(np.stack([np.asarray(c.T_cw, np.float32) for c in scene.cameras])).to(dev)
    return params, cams, viewmats.contiguous()


def gpu_forward(scene: Scene, tile=16, rast=None):
    rast = rast or R.GaussianRasterizer(tile)
    params, cams, vm = to_device(scene)
    color, depth, alpha, ws = rast.render_forward(params, scene.sh_degree, cams, vm)
    torch.cuda.synchronize()
    out = []
    for c, d, a in zip(R.split_views(color, cams, 3), R.split_views(depth, cams), R.split_views(alpha, cams)):
        out.append(dict(color=c.cpu().numpy().astype(np.float64), depth=d.cpu().numpy().astype(np.float64),
                        alpha=a.cpu().numpy().astype(np.float64)))
    return out, (rast, params, cams, vm, ws, color, depth, alpha)


def upstream(scene: Scene, seed=5):
    """Random upstream gradients (per view [3,H,W], [H,W], [H,W])."""
    rng = np.random.default_rng(seed)
    gC = [rng.uniform(-1, 1, (3, c.H, c.W)) for c in scene.cameras]
    gD = [rng.uniform(-1, 1, (c.H, c.W)) * 0.1 for c in scene.cameras]
    gA = [rng.uniform(-1, 1, (c.H, c.W)) for c in scene.cameras]
    return gC, gD, gA


def gpu_backward(scene: Scene, state, gC, gD, gA):
    rast, params, cams, vm, ws, color, depth, alpha = state
    dev = color.device
    flat = lambda arrs: torch.from_numpy(np.concatenate([np.asarray(a, np.float32).reshape(-1) for a in arrs])).to(dev)
    dC, dD, dA = flat(gC), flat(gD), flat(gA)
    grads = {k: torch.empty_like(v) for k, v in params.items()}
    d_pose = torch.empty(len(cams), 6, device=dev)
    rast.backward_raw(params, scene.sh_degree, cams, vm, ws, dC, dD, dA, grads, d_pose)
    torch.cuda.synchronize()
    out = {k: v.cpu().numpy().astype(np.float64) for k, v in grads.items()}
    out["pose"] = d_pose.cpu().numpy().astype(np.float64)
    return out


def near_threshold(ref):
    """Pixels where a decision of the oracle lies within FP32 reach of its
    threshold (see MARGIN, ZMARGIN)."""
    return (ref["margin"] < MARGIN) | (ref["zmargin"] < ZMARGIN)


def compare_images(ref, got, label=""):
    """Checks one view; returns (n_flip_pixels, n_pixels, max errors dict)."""
    dC = np.abs(got["color"] - ref["color"]).max(axis=0)
    dD = np.abs(got["depth"] - ref["depth"]) / np.maximum(np.abs(ref["depth"]), 1e-3)
    dA = np.abs(got["alpha"] - ref["alpha"])
    bad = (dC > COLOR_TOL) | (dD > DEPTH_TOL) | (dA > ALPHA_TOL)
    flip = near_threshold(ref)
    hard = bad & ~flip
    errs = dict(color=float(dC.max()), depth=float(dD.max()), alpha=float(dA.max()),
                color_nonflip=float(dC[~flip].max()) if (~flip).any() else 0.0,
                near_threshold=int(flip.sum()))
    assert not hard.any(), (
        f"{label}: {int(hard.sum())} pixels out of tolerance away from every threshold; "
        f"worst colour {dC[~flip].max():.3g}, depth {dD[~flip].max():.3g}, alpha {dA[~flip].max():.3g}")
    return int((bad & flip).sum()), int(bad.size), errs


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def compare_grads(ref: dict, got: dict, keys=("means", "log_scales", "quats", "opacity_logits", "sh", "pose"),
                  tol=GRAD_TOL, label=""):
    errs = {k: rel_l2(got[k], ref[k]) for k in keys}
    bad = {k: e for k, e in errs.items() if not e <= tol}
    assert not bad, f"{label}: gradient relative L2 above {tol}: {bad}"
    return errs
