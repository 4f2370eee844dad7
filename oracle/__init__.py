"""FP64 CPU oracle of the differentiable Gaussian rasteriser (test infrastructure).

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline leg may
import this package.  It shares no code with the CUDA library: the C source
next to this file (gsr_oracle.c) restates the paper's rendering equation
(Sec. 3.3, Eq. "rendering") and its backward in FP64, and this module only
marshals numpy arrays into it.

Parity is pinned in tests/test_oracle_pins.py against closed forms,
quadrature, library routines, brute force and finite differences.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import List, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gsr_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libgsr_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into oracle/_build/."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared", "-o", tmp,
                               _SRC, "-lm", "-lpthread"])
        os.replace(tmp, _LIB)
    return _LIB


class _Gaussians(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("sh_degree", ctypes.c_int),
                ("means", ctypes.c_void_p), ("log_scales", ctypes.c_void_p),
                ("quats", ctypes.c_void_p), ("opacity_logits", ctypes.c_void_p),
                ("sh", ctypes.c_void_p)]


class _Camera(ctypes.Structure):
    _fields_ = [("H", ctypes.c_int), ("W", ctypes.c_int),
                ("fx", ctypes.c_double), ("fy", ctypes.c_double),
                ("cx", ctypes.c_double), ("cy", ctypes.c_double),
                ("T_cw", ctypes.c_double * 12)]


def _load():
    global _lib
    if _lib is None:
        build()
        _lib = ctypes.CDLL(_LIB)
        for name in ("og_render", "og_render_backward", "og_project", "og_sh_basis", "og_quat_to_rot"):
            getattr(_lib, name).restype = ctypes.c_int
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


class _Packed:
    """float64 copies of a scene's parameters and cameras, kept alive for a call."""

    def __init__(self, scene, cameras=None):
        self.arrays = [np.ascontiguousarray(np.asarray(a, dtype=np.float64)) for a in
                       (scene.means, scene.log_scales, scene.quats, scene.opacity_logits, scene.sh)]
        self.g = _Gaussians(int(scene.means.shape[1]), int(scene.sh_degree),
                            *[a.ctypes.data for a in self.arrays])
        cams = scene.cameras if cameras is None else cameras
        self.V = len(cams)
        self.cams = (_Camera * max(self.V, 1))()
        for i, c in enumerate(cams):
            self.cams[i].H, self.cams[i].W = int(c.H), int(c.W)
            self.cams[i].fx, self.cams[i].fy = float(c.fx), float(c.fy)
            self.cams[i].cx, self.cams[i].cy = float(c.cx), float(c.cy)
            T = np.asarray(c.T_cw, dtype=np.float64).reshape(12)
            for k in range(12):
                self.cams[i].T_cw[k] = float(T[k])
        self.sizes = [(int(c.H), int(c.W)) for c in cams]


def _pixels(packed: _Packed, pixels):
    if pixels is None:
        counts = [h * w for h, w in packed.sizes]
        return None, None, counts
    counts = [len(p) for p in pixels]
    off = np.zeros(len(counts) + 1, dtype=np.int64)
    off[1:] = np.cumsum(counts)
    flat = np.ascontiguousarray(np.concatenate([np.asarray(p, dtype=np.int64) for p in pixels])
                                if counts else np.zeros(0, np.int64))
    return off, flat, counts


def _split(flat, counts, sizes, full, tail_shape):
    out, base = [], 0
    for n, (h, w) in zip(counts, sizes):
        a = flat[base:base + n]
        if full:
            a = a.reshape((h, w) + tail_shape)
        out.append(a)
        base += n
    return out


# per pixel: r, g, b, depth, opacity, T_final, threshold margin, median depth, median margin,
# depth-order margin
_NOUT = 10


def _pixel_dict(o, n):
    return dict(color=np.moveaxis(o[..., 0:3], -1, 0), depth=o[..., 3], alpha=o[..., 4], T=o[..., 5],
                margin=o[..., 6], median_depth=o[..., 7], median_margin=o[..., 8], zmargin=o[..., 9],
                ncontrib=n)


def render(scene, pixels: Optional[Sequence[np.ndarray]] = None, brute: bool = False,
           threads: int = 0, cameras=None):
    """Forward render.  pixels: per view arrays of linear indices y*W+x (None
    = all).  Returns per view dicts with color [3,...], depth, alpha, T,
    ncontrib, margin (cutoff, alpha-skip and stop decisions), zmargin
    (depth-order decisions), median_depth, median_margin (full images are
    [H, W])."""
    lib = _load()
    pk = _Packed(scene, cameras)
    off, flat, counts = _pixels(pk, pixels)
    P = int(sum(counts))
    out = np.zeros((max(P, 1), _NOUT), np.float64)
    nc = np.zeros(max(P, 1), np.int32)
    lib.og_render(ctypes.byref(pk.g), pk.V, pk.cams,
                  None if off is None else _ptr(off), None if flat is None else _ptr(flat),
                  int(brute), int(threads), _ptr(out), _ptr(nc))
    full = pixels is None
    res = []
    outs = _split(out[:P], counts, pk.sizes, full, (_NOUT,))
    ncs = _split(nc[:P], counts, pk.sizes, full, ())
    for o, n in zip(outs, ncs):
        res.append(_pixel_dict(o, n))
    return res


def render_backward(scene, gC: List[np.ndarray], gD: List[np.ndarray], gA: List[np.ndarray],
                    pixels: Optional[Sequence[np.ndarray]] = None, brute: bool = False,
                    threads: int = 0, want_screen: bool = False, cameras=None,
                    gM: Optional[List[np.ndarray]] = None):
    """Forward + backward with upstream grads per view: gC [3, ...], gD, gA
    (and optionally gM, dL/d median depth) shaped like the selected pixels
    ([3,H,W]/[H,W] for full images, [3,n]/[n] for pixel lists).  Returns
    (per view forward dicts, grads dict)."""
    lib = _load()
    pk = _Packed(scene, cameras)
    off, flat, counts = _pixels(pk, pixels)
    P = int(sum(counts))
    gCf = np.ascontiguousarray(np.concatenate(
        [np.moveaxis(np.asarray(g, np.float64).reshape(3, -1), 0, -1) for g in gC]) if P else np.zeros((1, 3)))
    gDf = np.ascontiguousarray(np.concatenate([np.asarray(g, np.float64).reshape(-1) for g in gD]) if P else np.zeros(1))
    gAf = np.ascontiguousarray(np.concatenate([np.asarray(g, np.float64).reshape(-1) for g in gA]) if P else np.zeros(1))
    gMf = None if gM is None else np.ascontiguousarray(
        np.concatenate([np.asarray(g, np.float64).reshape(-1) for g in gM]) if P else np.zeros(1))
    N = scene.means.shape[1]
    K = (scene.sh_degree + 1) ** 2
    out = np.zeros((max(P, 1), _NOUT), np.float64)
    nc = np.zeros(max(P, 1), np.int32)
    gm = np.zeros((3, N)); gls = np.zeros((3, N)); gq = np.zeros((4, N)); gl = np.zeros(N)
    gsh = np.zeros((3 * K, N)); pose = np.zeros((pk.V, 6))
    screen = np.zeros((pk.V, 10, N)) if want_screen else None
    lib.og_render_backward(ctypes.byref(pk.g), pk.V, pk.cams,
                           None if off is None else _ptr(off), None if flat is None else _ptr(flat),
                           int(brute), int(threads), _ptr(gCf), _ptr(gDf), _ptr(gAf),
                           None if gMf is None else _ptr(gMf), _ptr(out), _ptr(nc),
                           _ptr(gm), _ptr(gls), _ptr(gq), _ptr(gl), _ptr(gsh), _ptr(pose),
                           None if screen is None else _ptr(screen))
    full = pixels is None
    res = []
    for o, n in zip(_split(out[:P], counts, pk.sizes, full, (_NOUT,)), _split(nc[:P], counts, pk.sizes, full, ())):
        res.append(_pixel_dict(o, n))
    grads = dict(means=gm, log_scales=gls, quats=gq, opacity_logits=gl, sh=gsh, pose=pose)
    if want_screen:
        grads["screen"] = screen
    return res, grads


PROJ_FIELDS = ("valid", "u", "v", "z", "conic0", "conic1", "conic2", "cov0", "cov1", "cov2",
               "opacity", "r", "g", "b", "clamp_x", "clamp_y")


def project(scene, view: int = 0, camera=None):
    """Per-Gaussian projection into one view: dict of [N] arrays."""
    lib = _load()
    cams = [camera if camera is not None else scene.cameras[view]]
    pk = _Packed(scene, cams)
    N = scene.means.shape[1]
    out = np.zeros((max(N, 1), 16))
    lib.og_project(ctypes.byref(pk.g), pk.cams, _ptr(out))
    return {k: out[:N, i] for i, k in enumerate(PROJ_FIELDS)}


def sh_basis(degree: int, direction) -> np.ndarray:
    lib = _load()
    d = np.ascontiguousarray(np.asarray(direction, np.float64).reshape(3))
    Y = np.zeros(16)
    lib.og_sh_basis(int(degree), _ptr(d), _ptr(Y))
    return Y


def quat_to_rot(q) -> np.ndarray:
    lib = _load()
    qq = np.ascontiguousarray(np.asarray(q, np.float64).reshape(4))
    R = np.zeros(9)
    lib.og_quat_to_rot(_ptr(qq), _ptr(R))
    return R.reshape(3, 3)


def _quad_min_over_box(a, b, d, u, v, x0, x1, y0, y1):
    """min over the box [x0, x1] x [y0, y1] of the convex quadratic
    q(x, y) = a dx^2 + 2 b dx dy + d dy^2, (dx, dy) = (x - u, y - v): zero
    when the centre is inside, else the smallest of the four edges' 1-D
    minima (clamped stationary points)."""
    if x0 <= u <= x1 and y0 <= v <= y1:
        return 0.0
    best = np.inf
    for x in (x0, x1):          # vertical edges: minimise over y
        dx = x - u
        dy = min(max(-b * dx / d, y0 - v), y1 - v)
        best = min(best, a * dx * dx + 2 * b * dx * dy + d * dy * dy)
    for y in (y0, y1):          # horizontal edges: minimise over x
        dy = y - v
        dx = min(max(-b * dy / a, x0 - u), x1 - u)
        best = min(best, a * dx * dx + 2 * b * dx * dy + d * dy * dy)
    return best


def densify_stats(scene, screen, cameras=None):
    """Densification statistics of one batch of views (the adaptive density
    control of 3DGS that the paper's mapper uses, Sec. 3.3): per Gaussian,
      grad   = sum over views where it is visible of |(dL/du, dL/dv)| (pixels),
      count  = number of such views,
      radius = max over them of 3 sqrt(lambda_max(Sigma')) (pixels),
    with "visible" = not culled and its cutoff ellipse, d^2 <= min(9,
    2 ln(255 sigma)), meets the rectangle [0, W-1] x [0, H-1] spanned by the
    pixel centres.  screen: grads["screen"] of render_backward(...,
    want_screen=True).  Also returns margin, per Gaussian the smallest
    |min d^2 / d2max - 1| of its views' visibility decisions."""
    cams = scene.cameras if cameras is None else cameras
    N = scene.means.shape[1]
    grad, count, radius = np.zeros(N), np.zeros(N), np.zeros(N)
    margin = np.full(N, np.inf)
    for v, c in enumerate(cams):
        P = project(scene, camera=c)
        for g in range(N):
            if not P["valid"][g]:
                continue
            d2max = min(9.0, 2.0 * np.log(255.0 * P["opacity"][g]))
            if not d2max >= 0:
                continue
            qmin = _quad_min_over_box(P["conic0"][g], P["conic1"][g], P["conic2"][g], P["u"][g], P["v"][g],
                                      0.0, c.W - 1.0, 0.0, c.H - 1.0)
            margin[g] = min(margin[g], abs(qmin / max(d2max, 1e-300) - 1))
            if qmin > d2max:
                continue
            grad[g] += np.hypot(screen[v][0][g], screen[v][1][g])
            count[g] += 1
            c0, c1, c2 = P["cov0"][g], P["cov1"][g], P["cov2"][g]
            mid = 0.5 * (c0 + c2)
            lam = mid + np.sqrt(max(mid * mid - (c0 * c2 - c1 * c1), 0.0))
            radius[g] = max(radius[g], 3.0 * np.sqrt(lam))
    return dict(grad=grad, count=count, radius=radius, margin=margin)
