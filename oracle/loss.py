"""FP64 oracle of the mixed rendering loss, Eq. "rnd_loss" (Sec. 3.3) --
test infrastructure only.

    L_i = lambda1 [ (1 - lambda2) |I' - I*|_1 + lambda2 (1 - SSIM(I', I*)) ]
          + (1 - lambda1) |Z' - Z*|_1

Readings (the paper names the terms, following MonoGS/3DGS, without the
details): the L1 norms are means over pixels (colour: over the 3 channels
too); SSIM is the structural similarity of Wang et al. with an 11x11
Gaussian window of sigma 1.5, C1 = 0.01^2, C2 = 0.03^2, computed per channel
with zero padding ("same" size) and averaged over channels and pixels; the
loss of a keyframe window is the sum over its views.  lambda2 = 0.2 and
lambda1 = 0.9 / 0.8 (Supp. Sec. 1.2).

Plain PyTorch CPU ops in float64; gradients by autograd.
"""
from __future__ import annotations

import math

import numpy as np
import torch
import torch.nn.functional as F

WINDOW = 11
SIGMA = 1.5
C1 = 0.01 ** 2
C2 = 0.03 ** 2


def gaussian_1d(size: int = WINDOW, sigma: float = SIGMA) -> torch.Tensor:
    x = torch.arange(size, dtype=torch.float64) - (size // 2)
    g = torch.exp(-(x * x) / (2 * sigma * sigma))
    return g / g.sum()


def _blur(img: torch.Tensor) -> torch.Tensor:
    """Zero-padded 'same' correlation of [C, H, W] with the 2-D Gaussian window."""
    g = gaussian_1d()
    w2 = torch.outer(g, g)[None, None]
    C = img.shape[0]
    return F.conv2d(img[:, None], w2, padding=WINDOW // 2).reshape(C, img.shape[1], img.shape[2])


def ssim_map(x: torch.Tensor, y: torch.Tensor) -> torch.Tensor:
    """Per-pixel SSIM of two [C, H, W] float64 images."""
    mx, my = _blur(x), _blur(y)
    sxx = _blur(x * x) - mx * mx
    syy = _blur(y * y) - my * my
    sxy = _blur(x * y) - mx * my
    return ((2 * mx * my + C1) * (2 * sxy + C2)) / ((mx * mx + my * my + C1) * (sxx + syy + C2))


def view_loss(color, target_color, depth, target_depth, lambda1: float, lambda2: float):
    """Eq. "rnd_loss" of one view; depth terms are skipped when target_depth is None."""
    l1c = (color - target_color).abs().mean()
    s = ssim_map(color, target_color).mean()
    loss = lambda1 * ((1 - lambda2) * l1c + lambda2 * (1 - s))
    if target_depth is not None:
        loss = loss + (1 - lambda1) * (depth - target_depth).abs().mean()
    return loss


def window_loss_and_grads(colors, target_colors, depths, target_depths, lambda1: float, lambda2: float):
    """Sum over views; returns (loss, [dL/dcolor], [dL/ddepth]) as float64 numpy."""
    cs = [torch.tensor(np.asarray(c, np.float64), requires_grad=True) for c in colors]
    ds = [torch.tensor(np.asarray(d, np.float64), requires_grad=True) for d in depths]
    total = 0.0
    for c, tc, d, td in zip(cs, target_colors, ds, target_depths):
        tct = torch.tensor(np.asarray(tc, np.float64))
        tdt = None if td is None else torch.tensor(np.asarray(td, np.float64))
        total = total + view_loss(c, tct, d, tdt, lambda1, lambda2)
    total.backward()
    return (float(total), [c.grad.numpy() for c in cs],
            [d.grad.numpy() if d.grad is not None else np.zeros(d.shape) for d in ds])


def ssim_brute(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """Direct windowed SSIM of one channel [H, W]: explicit sums over the
    11x11 window, pixels outside the image counted as zero."""
    H, W = x.shape
    r = WINDOW // 2
    g = [math.exp(-(k - r) ** 2 / (2 * SIGMA ** 2)) for k in range(WINDOW)]
    s = sum(g)
    g = [v / s for v in g]
    out = np.zeros((H, W))
    for i in range(H):
        for j in range(W):
            mx = my = exx = eyy = exy = 0.0
            for a in range(WINDOW):
                for b in range(WINDOW):
                    ii, jj = i + a - r, j + b - r
                    if 0 <= ii < H and 0 <= jj < W:
                        w = g[a] * g[b]
                        xv, yv = x[ii, jj], y[ii, jj]
                        mx += w * xv
                        my += w * yv
                        exx += w * xv * xv
                        eyy += w * yv * yv
                        exy += w * xv * yv
            sx, sy, sxy = exx - mx * mx, eyy - my * my, exy - mx * my
            out[i, j] = ((2 * mx * my + C1) * (2 * sxy + C2)) / ((mx * mx + my * my + C1) * (sx + sy + C2))
    return out
