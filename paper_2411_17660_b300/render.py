"""PyTorch front end of the rasteriser: tensors in, tensors out.

torch provides device memory and the stream; all arithmetic runs in
libgsr.so.  `GaussianRasterizer.render` is differentiable through
`torch.autograd.Function` with gradients for every Gaussian parameter and a
per-view pose tangent (Sec. 3.3 of the paper: the map is "optimized via
backpropagation" and keyframe poses can be finetuned with the rendering
objective).

Pose convention: each view has T_cw = [W | t] (world -> camera, float32
[V, 3, 4] on the device).  The differentiable pose input is a tangent
xi = (rho, phi) in R^6 per view for the left perturbation Exp(xi) T_cw; the
renderer always renders at xi = 0 and returns dL/dxi there.  After an
optimiser step the caller folds xi into T_cw and resets it to zero.
"""
from __future__ import annotations

import ctypes
import dataclasses
from typing import List, Optional, Sequence

import torch

from . import binding as _b


@dataclasses.dataclass(frozen=True)
class Intrinsics:
    H: int
    W: int
    fx: float
    fy: float
    cx: float
    cy: float


PARAM_NAMES = ("means", "log_scales", "quats", "opacity_logits", "sh")


def _check_param(name, t: torch.Tensor, rows: int, N: int):
    if not t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous float32 CUDA tensor")
    shape = (N,) if rows == 0 else (rows, N)
    if tuple(t.shape) != shape:
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {shape}")


def gaussians_struct(means, log_scales, quats, opacity_logits, sh, sh_degree: int) -> _b.Gaussians:
    N = int(means.shape[1])
    K = (sh_degree + 1) ** 2
    _check_param("means", means, 3, N)
    _check_param("log_scales", log_scales, 3, N)
    _check_param("quats", quats, 4, N)
    _check_param("opacity_logits", opacity_logits, 0, N)
    _check_param("sh", sh, 3 * K, N)
    return _b.Gaussians(N, sh_degree, means.data_ptr(), log_scales.data_ptr(), quats.data_ptr(),
                        opacity_logits.data_ptr(), sh.data_ptr())


def pixel_offsets(cams: Sequence[Intrinsics]) -> List[int]:
    off, o = [], 0
    for c in cams:
        off.append(o)
        o += c.H * c.W
    off.append(o)
    return off


def view_structs(cams, viewmats: torch.Tensor, color=None, depth=None, alpha=None,
                 median_depth=None) -> List[_b.View]:
    """C view structs; color/depth/alpha/median_depth are flat buffers of all
    views (colour [3*P_v] per view, laid out view after view)."""
    if viewmats.dtype != torch.float32 or not viewmats.is_cuda or not viewmats.is_contiguous() or \
            tuple(viewmats.shape) != (len(cams), 3, 4):
        raise ValueError("viewmats must be a contiguous float32 CUDA tensor [V, 3, 4]")
    off = pixel_offsets(cams)
    out = []
    base = viewmats.data_ptr()
    for v, c in enumerate(cams):
        out.append(_b.View(
            int(c.H), int(c.W), float(c.fx), float(c.fy), float(c.cx), float(c.cy), base + 48 * v,
            0 if color is None else color.data_ptr() + 4 * 3 * off[v],
            0 if depth is None else depth.data_ptr() + 4 * off[v],
            0 if alpha is None else alpha.data_ptr() + 4 * off[v],
            0 if median_depth is None else median_depth.data_ptr() + 4 * off[v]))
    return out


def split_views(flat: torch.Tensor, cams, channels: int = 1):
    """Per-view [C, H, W] (or [H, W]) views of a flat output buffer."""
    off = pixel_offsets(cams)
    res = []
    for v, c in enumerate(cams):
        a = flat[channels * off[v]:channels * off[v + 1]]
        res.append(a.view(channels, c.H, c.W) if channels > 1 else a.view(c.H, c.W))
    return res


class GaussianRasterizer:
    """Batched differentiable Gaussian rasteriser over a keyframe window."""

    def __init__(self, tile: int = 16, spin_limit: int = 0, flags: int = 0, binning: str = "tile", batch: int = 32,
                 fwd_rows: int = 0):
        if binning not in ("tile", "radix"):
            raise ValueError(f"binning must be 'tile' or 'radix', not {binning!r}")
        self.ctx = _b.Context(tile, spin_limit, flags, _b.BIN_TILE if binning == "tile" else _b.BIN_RADIX, batch,
                              fwd_rows)
        self.tile = tile
        self.binning = binning
        self.batch = batch
        self.fwd_rows = fwd_rows or (8 if tile == 8 else 16)
        self._cap_hint = {}

    # ------------------------------------------------------------ workspace
    def workspace_bytes(self, N: int, cams, key_capacity: int = 0) -> int:
        dummy = [_b.View(c.H, c.W, c.fx, c.fy, c.cx, c.cy, 1, 1, 0, 0, 0) for c in cams]
        return self.ctx.workspace_size(N, dummy, key_capacity)

    def alloc_workspace(self, N: int, cams, key_capacity: int = 0, device=None) -> torch.Tensor:
        nbytes = self.workspace_bytes(N, cams, key_capacity)
        return torch.empty(nbytes, dtype=torch.uint8, device=device or torch.device("cuda"))

    def info(self, ws: torch.Tensor) -> _b.Info:
        return self.ctx.read_info(ws.data_ptr(), ws.numel(), torch.cuda.current_stream().cuda_stream)

    # ------------------------------------------------------------ raw calls
    def forward_raw(self, params, sh_degree: int, cams, viewmats: torch.Tensor, ws: torch.Tensor,
                    color: torch.Tensor, depth: Optional[torch.Tensor], alpha: Optional[torch.Tensor],
                    median_depth: Optional[torch.Tensor] = None):
        g = gaussians_struct(*[params[k] for k in PARAM_NAMES], sh_degree)
        views = view_structs(cams, viewmats, color, depth, alpha, median_depth)
        st = self.ctx.render(g, views, ws.data_ptr(), ws.numel(), torch.cuda.current_stream().cuda_stream)
        self.ctx.check(st, "gsr_render")

    def forward_l1_raw(self, params, sh_degree: int, cams, viewmats: torch.Tensor, ws: torch.Tensor,
                       color: torch.Tensor, depth: Optional[torch.Tensor], alpha: Optional[torch.Tensor],
                       target_color, target_depth, color_weight: float, depth_weight: float, d_color, d_depth,
                       loss, median_depth: Optional[torch.Tensor] = None):
        """forward_raw and l1_loss in one call (gsr_render_l1): the forward
        blend also writes d_color, d_depth and the device scalar loss."""
        g = gaussians_struct(*[params[k] for k in PARAM_NAMES], sh_degree)
        views = view_structs(cams, viewmats, color, depth, alpha, median_depth)
        t = l1_views(cams, target_color, target_depth, d_color, d_depth)
        st = self.ctx.render_l1(g, views, t, color_weight, depth_weight, loss.data_ptr(), ws.data_ptr(), ws.numel(),
                                torch.cuda.current_stream().cuda_stream)
        self.ctx.check(st, "gsr_render_l1")

    def backward_raw(self, params, sh_degree: int, cams, viewmats: torch.Tensor, ws: torch.Tensor,
                     d_color, d_depth, d_alpha, grads: dict, d_pose: Optional[torch.Tensor], accumulate=False,
                     d_median_depth: Optional[torch.Tensor] = None, densify: Optional[dict] = None):
        """densify: optional dict of [N] float32 tensors grad, count, radius that
        receive the densification statistics of the batch (accumulated like
        the gradients when accumulate is set)."""
        g = gaussians_struct(*[params[k] for k in PARAM_NAMES], sh_degree)
        views = view_structs(cams, viewmats)
        off = pixel_offsets(cams)
        vg = []
        for v in range(len(cams)):
            vg.append(_b.ViewGrad(
                0 if d_color is None else d_color.data_ptr() + 4 * 3 * off[v],
                0 if d_depth is None else d_depth.data_ptr() + 4 * off[v],
                0 if d_alpha is None else d_alpha.data_ptr() + 4 * off[v],
                0 if d_median_depth is None else d_median_depth.data_ptr() + 4 * off[v],
                0 if d_pose is None else d_pose.data_ptr() + 4 * 6 * v))
        dens = [0, 0, 0] if densify is None else [densify[k].data_ptr() for k in ("grad", "count", "radius")]
        out = _b.Grads(*[grads[k].data_ptr() for k in PARAM_NAMES], int(accumulate), *dens)
        st = self.ctx.render_backward(g, views, vg, out, ws.data_ptr(), ws.numel(),
                                      torch.cuda.current_stream().cuda_stream)
        self.ctx.check(st, "gsr_render_backward")

    # ------------------------------------------------------------ surfels (2DGS)
    def surfels_forward_raw(self, params, sh_degree: int, cams, viewmats: torch.Tensor, ws: torch.Tensor,
                            color: torch.Tensor, depth=None, alpha=None, normal=None, distortion=None):
        """Surfel render into flat buffers (normal: [3 * P_v] per view like colour)."""
        g = gaussians_struct(*[params[k] for k in PARAM_NAMES], sh_degree)
        views = view_structs(cams, viewmats, color, depth, alpha)
        off = pixel_offsets(cams)
        extra = [_b.SurfelOut(0 if normal is None else normal.data_ptr() + 4 * 3 * off[v],
                              0 if distortion is None else distortion.data_ptr() + 4 * off[v])
                 for v in range(len(cams))]
        st = self.ctx.render_surfels(g, views, extra, ws.data_ptr(), ws.numel(),
                                     torch.cuda.current_stream().cuda_stream)
        self.ctx.check(st, "gsr_render_surfels")

    def surfels_backward_raw(self, params, sh_degree: int, cams, viewmats: torch.Tensor, ws: torch.Tensor,
                             d_color, d_depth, d_alpha, d_normal, d_distortion, grads: dict,
                             d_pose: Optional[torch.Tensor], accumulate=False):
        g = gaussians_struct(*[params[k] for k in PARAM_NAMES], sh_degree)
        views = view_structs(cams, viewmats)
        off = pixel_offsets(cams)
        ptr = lambda t, v, ch: 0 if t is None else t.data_ptr() + 4 * ch * off[v]
        vg = [_b.ViewGrad(ptr(d_color, v, 3), ptr(d_depth, v, 1), ptr(d_alpha, v, 1), 0,
                          0 if d_pose is None else d_pose.data_ptr() + 4 * 6 * v) for v in range(len(cams))]
        extra = [_b.SurfelGrad(ptr(d_normal, v, 3), ptr(d_distortion, v, 1)) for v in range(len(cams))]
        out = _b.Grads(*[grads[k].data_ptr() for k in PARAM_NAMES], int(accumulate), 0, 0, 0)
        st = self.ctx.render_surfels_backward(g, views, vg, extra, out, ws.data_ptr(), ws.numel(),
                                              torch.cuda.current_stream().cuda_stream)
        self.ctx.check(st, "gsr_render_surfels_backward")

    # ------------------------------------------------------------ convenience
    def render_forward(self, params, sh_degree: int, cams, viewmats: torch.Tensor,
                       ws: Optional[torch.Tensor] = None, grow: bool = True):
        """Forward render; allocates (and, when grow, resizes) the workspace
        from the key count the device reports.  Returns (color, depth, alpha, ws)
        as flat buffers."""
        N = int(params["means"].shape[1])
        P = pixel_offsets(cams)[-1]
        dev = params["means"].device
        color = torch.empty(3 * P, dtype=torch.float32, device=dev)
        depth = torch.empty(P, dtype=torch.float32, device=dev)
        alpha = torch.empty(P, dtype=torch.float32, device=dev)
        key = (N, tuple(cams))
        if ws is None:
            ws = self.alloc_workspace(N, cams, self._cap_hint.get(key, 0), dev)
        for _ in range(4):
            self.forward_raw(params, sh_degree, cams, viewmats, ws, color, depth, alpha)
            if not grow:
                break
            inf = self.info(ws)
            if inf.status == _b.OK:
                break
            if inf.status != _b.ECAPACITY:
                raise _b.GsrError(inf.status, "device error in gsr_render")
            cap = int(inf.keys * 1.25) + 4096
            self._cap_hint[key] = cap
            ws = self.alloc_workspace(N, cams, cap, dev)
        return color, depth, alpha, ws

    def render(self, means, log_scales, quats, opacity_logits, sh, sh_degree: int, cams,
               viewmats: torch.Tensor, pose_tangent: Optional[torch.Tensor] = None):
        """Differentiable render of the batch.  Returns flat (color, depth,
        alpha); split them with split_views."""
        if pose_tangent is None:
            pose_tangent = torch.zeros(len(cams), 6, device=means.device)
        return _RenderFn.apply(self, tuple(cams), viewmats, sh_degree, means, log_scales, quats,
                               opacity_logits, sh, pose_tangent)


class _RenderFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, rast, cams, viewmats, sh_degree, means, log_scales, quats, opacity_logits, sh, pose_tangent):
        params = dict(means=means.detach(), log_scales=log_scales.detach(), quats=quats.detach(),
                      opacity_logits=opacity_logits.detach(), sh=sh.detach())
        color, depth, alpha, ws = rast.render_forward(params, sh_degree, list(cams), viewmats)
        ctx.rast, ctx.cams, ctx.sh_degree, ctx.ws = rast, list(cams), sh_degree, ws
        ctx.save_for_backward(means, log_scales, quats, opacity_logits, sh, viewmats)
        return color, depth, alpha

    @staticmethod
    def backward(ctx, d_color, d_depth, d_alpha):
        means, log_scales, quats, opacity_logits, sh, viewmats = ctx.saved_tensors
        params = dict(means=means, log_scales=log_scales, quats=quats, opacity_logits=opacity_logits, sh=sh)
        grads = {k: torch.empty_like(v) for k, v in params.items()}
        d_pose = torch.empty(len(ctx.cams), 6, dtype=torch.float32, device=means.device)
        cont = lambda t: None if t is None else t.contiguous()
        ctx.rast.backward_raw(params, ctx.sh_degree, ctx.cams, viewmats, ctx.ws, cont(d_color), cont(d_depth),
                              cont(d_alpha), grads, d_pose)
        return (None, None, None, None, grads["means"], grads["log_scales"], grads["quats"],
                grads["opacity_logits"], grads["sh"], d_pose)


def l1_views(cams, target_color, target_depth, d_color, d_depth):
    """The per-view gsr_l1_view structs of flat target / gradient buffers laid
    out like the render outputs."""
    off = pixel_offsets(cams)
    t = []
    for v in range(len(cams)):
        t.append(_b.L1View(target_color.data_ptr() + 12 * off[v],
                           0 if target_depth is None else target_depth.data_ptr() + 4 * off[v],
                           d_color.data_ptr() + 12 * off[v],
                           0 if d_depth is None else d_depth.data_ptr() + 4 * off[v]))
    return t


def l1_loss(rast: GaussianRasterizer, cams, viewmats, color, depth, target_color, target_depth,
            color_weight: float, depth_weight: float, d_color, d_depth, loss):
    """L1 colour + depth loss (library kernel): fills d_color, d_depth and the
    device scalar loss.  All arguments are flat buffers laid out like the
    render outputs."""
    views = view_structs(cams, viewmats, color, depth, None)
    t = l1_views(cams, target_color, target_depth, d_color, d_depth)
    rast.ctx.l1_loss(views, t, color_weight, depth_weight, loss.data_ptr(), torch.cuda.current_stream().cuda_stream)


def rgbd_loss(rast: GaussianRasterizer, cams, viewmats, color, depth, target_color, target_depth,
              lambda1: float, lambda2: float, d_color, d_depth, loss):
    """Mixed L1 + SSIM colour and L1 depth loss of the paper (library kernel):
    fills d_color, d_depth and the device scalar loss.  Flat buffers laid out
    like the render outputs; lambda2 = 0.2 and lambda1 = 0.9 / 0.8 in the paper."""
    views = view_structs(cams, viewmats, color, depth, None)
    off = pixel_offsets(cams)
    t = []
    for v in range(len(cams)):
        t.append(_b.L1View(target_color.data_ptr() + 12 * off[v],
                           0 if target_depth is None else target_depth.data_ptr() + 4 * off[v],
                           d_color.data_ptr() + 12 * off[v],
                           0 if d_depth is None else d_depth.data_ptr() + 4 * off[v]))
    rast.ctx.rgbd_loss(views, t, lambda1, lambda2, loss.data_ptr(), torch.cuda.current_stream().cuda_stream)
