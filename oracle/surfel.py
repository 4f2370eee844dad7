"""FP64 oracle of the 2-D surfel ("2DGS") rasteriser the paper compares its
3-D Gaussians with (Sec. 3.3, last paragraph; Supp. "2D Gaussian
Splatting") -- test infrastructure only.

Plain PyTorch CPU ops in float64; gradients by autograd, pose gradients
through the left perturbation T_cw <- (I + xi^) T_cw at xi = 0.

Readings (the paper cites 2DGS for the representation and its two extra
losses without restating them):
  * a surfel is a flat disk: centre mu, tangents t_u, t_v (first two columns
    of R(q)), scales s_u = exp(log_s0), s_v = exp(log_s1) (log_s2 unused),
    normal t_w (third column), opacity sigma, SH colour as for 3-D Gaussians;
  * with a = s_u W t_u, b = s_v W t_v, p = W mu + t (camera frame) and the
    pinhole K, the homography M = K [a | b | p] maps disk coordinates
    (u, v, 1) to homogeneous pixels; a pixel (x, y) meets the disk where the
    planes h_x = M_0 - x M_2 and h_y = M_1 - y M_2 cross:
    (u, v, 1) ~ h_x x h_y, and rho3 = u^2 + v^2;
  * low-pass fallback: rho2 = 2 |(x, y) - c|^2 (a screen-space Gaussian of
    variance 1/2 around the projected centre c); rho = min(rho3, rho2);
  * alpha = min(0.99, sigma exp(-rho / 2)), skipped when rho > 9 or
    alpha < 1/255, the walk stopping before T would drop below 1e-4;
    Gaussians are sorted by the depth p_z of their centre (then index);
  * culled: p_z <= 0.2, or the cutoff disk u^2 + v^2 <= 9 reaching the near
    plane (p_z - 3 sqrt(a_z^2 + b_z^2) <= 0.2), or 255 sigma < 1;
  * per pixel the oracle also reports a margin: the smallest relative
    distance of a threshold decision (as for 3-D Gaussians) or 0.1 sin(theta)
    of a contributor's ray-disk intersection (the 2x2 solve's conditioning);
  * outputs: colour, depth D = sum w z (z = a_z u + b_z v + p_z, the depth
    of the ray-disk intersection, where rho3 <= rho2; the centre's depth p_z
    where the low-pass term decides alpha, so that a grazing or missed disk
    never reports the depth of a far or backward intersection), opacity
    A = sum w, normal map
    N = sum w n (n = W t_w turned to face the camera, camera frame) and the
    depth distortion sum_{i > j} w_i w_j (z_i - z_j)^2.
"""
from __future__ import annotations

import math
from typing import List, Optional

import numpy as np
import torch

NEAR_Z = 0.2
CUTOFF = 9.0
ALPHA_MIN = 1.0 / 255.0
ALPHA_MAX = 0.99
T_STOP = 1e-4
LOWPASS = 2.0   # rho2 = LOWPASS |pixel - centre|^2


def sh_basis_t(deg: int, d: torch.Tensor) -> torch.Tensor:
    """Real SH (Condon-Shortley phase, order (l, m = -l..l)) of unit
    directions d [..., 3]; returns [..., (deg+1)^2]."""
    x, y, z = d[..., 0], d[..., 1], d[..., 2]
    pi = math.pi
    out = [torch.full_like(x, 0.5 * math.sqrt(1 / pi))]
    if deg >= 1:
        k1 = math.sqrt(3 / (4 * pi))
        out += [-k1 * y, k1 * z, -k1 * x]
    if deg >= 2:
        k2a, k2b, k2c = 0.5 * math.sqrt(15 / pi), 0.25 * math.sqrt(5 / pi), 0.25 * math.sqrt(15 / pi)
        out += [k2a * x * y, -k2a * y * z, k2b * (3 * z * z - 1), -k2a * x * z, k2c * (x * x - y * y)]
    if deg >= 3:
        k3a, k3b = 0.25 * math.sqrt(35 / (2 * pi)), 0.5 * math.sqrt(105 / pi)
        k3c, k3d, k3e = 0.25 * math.sqrt(21 / (2 * pi)), 0.25 * math.sqrt(7 / pi), 0.25 * math.sqrt(105 / pi)
        out += [-k3a * (3 * x * x * y - y ** 3), k3b * x * y * z, -k3c * y * (5 * z * z - 1),
                k3d * (5 * z ** 3 - 3 * z), -k3c * x * (5 * z * z - 1), k3e * z * (x * x - y * y),
                -k3a * (x ** 3 - 3 * x * y * y)]
    return torch.stack(out, -1)


def quat_to_rot_t(q: torch.Tensor) -> torch.Tensor:
    """Rotation matrices [N, 3, 3] of the normalised quaternions q [N, 4] (w, x, y, z)."""
    q = q / q.norm(dim=-1, keepdim=True)
    w, x, y, z = q.unbind(-1)
    return torch.stack([
        torch.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
        torch.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
        torch.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1)], -2)


def _hat(v):
    z = torch.zeros((), dtype=v.dtype)
    return torch.stack([torch.stack([z, -v[2], v[1]]), torch.stack([v[2], z, -v[0]]),
                        torch.stack([-v[1], v[0], z])])


def _view(P, cam, xi, sh_degree):
    """Per-surfel quantities of one view (autograd graph kept)."""
    T = torch.tensor(np.asarray(cam.T_cw, np.float64).reshape(3, 4))
    W, t = T[:, :3], T[:, 3]
    if xi is not None:   # left perturbation (I + xi^) T_cw, exact to first order at xi = 0
        W = W + _hat(xi[3:]) @ W
        t = t + _hat(xi[3:]) @ t + xi[:3]
    mu = P["means"].T                                        # [N, 3]
    R = quat_to_rot_t(P["quats"].T)                          # [N, 3, 3]
    su, sv = torch.exp(P["log_scales"][0]), torch.exp(P["log_scales"][1])
    pc = mu @ W.T + t
    a = su[:, None] * (R[:, :, 0] @ W.T)
    b = sv[:, None] * (R[:, :, 1] @ W.T)
    n = R[:, :, 2] @ W.T
    with torch.no_grad():
        flip = ((n * pc).sum(-1) > 0).double() * -2 + 1
    n = n * flip[:, None]
    sigma = torch.sigmoid(P["opacity_logits"])
    C = -(W.T @ t)
    dvec = mu - C
    Y = sh_basis_t(sh_degree, dvec / dvec.norm(dim=-1, keepdim=True))     # [N, K]
    K = (sh_degree + 1) ** 2
    sh = P["sh"].reshape(K, 3, -1).permute(2, 0, 1)                       # [N, K, 3]
    rgb = torch.clamp((Y[:, :, None] * sh).sum(1) + 0.5, min=0.0)
    fx, fy, cx, cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    M0 = fx * torch.stack([a[:, 0], b[:, 0], pc[:, 0]], -1) + cx * torch.stack([a[:, 2], b[:, 2], pc[:, 2]], -1)
    M1 = fy * torch.stack([a[:, 1], b[:, 1], pc[:, 1]], -1) + cy * torch.stack([a[:, 2], b[:, 2], pc[:, 2]], -1)
    M2 = torch.stack([a[:, 2], b[:, 2], pc[:, 2]], -1)
    with torch.no_grad():
        zmin = pc[:, 2] - 3.0 * torch.sqrt(a[:, 2] ** 2 + b[:, 2] ** 2)
        valid = (pc[:, 2] > NEAR_Z) & (zmin > NEAR_Z) & (255.0 * sigma >= 1.0)
    return dict(M0=M0, M1=M1, M2=M2, pc=pc, n=n, rgb=rgb, sigma=sigma, valid=valid, a=a, b=b)


def _composite(S, xs, ys):
    """Front-to-back compositing of the pixels (xs, ys) [P]; returns outputs
    [P] (colour [P, 3], normal [P, 3]) and per-pixel decision margins."""
    M0, M1, M2 = S["M0"], S["M1"], S["M2"]
    order = torch.from_numpy(np.lexsort((np.arange(M2.shape[0]), S["pc"][:, 2].detach().numpy())))
    M0, M1, M2 = M0[order], M1[order], M2[order]
    valid, sigma, rgb, n = S["valid"][order], S["sigma"][order], S["rgb"][order], S["n"][order]
    a, b, pc = S["a"][order], S["b"][order], S["pc"][order]
    x, y = xs[:, None, None], ys[:, None, None]
    hx = M0[None] - x * M2[None]
    hy = M1[None] - y * M2[None]
    q = torch.cross(hx, hy, dim=-1)                                     # [P, N, 3]
    u, v = q[..., 0] / q[..., 2], q[..., 1] / q[..., 2]
    rho3 = u * u + v * v
    cxy0, cxy1 = M0[:, 2] / M2[:, 2], M1[:, 2] / M2[:, 2]
    rho2 = LOWPASS * ((xs[:, None] - cxy0[None]) ** 2 + (ys[:, None] - cxy1[None]) ** 2)
    rho3 = torch.where(torch.isfinite(rho3), rho3, torch.full_like(rho3, math.inf))
    rho = torch.minimum(rho3, rho2)
    a_raw = sigma[None] * torch.exp(-0.5 * rho)
    # depth of the contributor: the ray-disk intersection where the disk term
    # decides alpha, the centre's depth where the screen-space low-pass does
    zint = torch.where(rho3 <= rho2, a[None, :, 2] * u + b[None, :, 2] * v + pc[None, :, 2],
                       pc[None, :, 2].expand_as(rho2))
    with torch.no_grad():
        keep = valid[None] & (rho <= CUTOFF) & (a_raw >= ALPHA_MIN)
        al = torch.where(keep, torch.clamp(a_raw, max=ALPHA_MAX), torch.zeros_like(a_raw))
        Tb = torch.cumprod(torch.cat([torch.ones_like(al[:, :1]), 1 - al[:, :-1]], 1), 1)
        stop = keep & (Tb * (1 - al) < T_STOP)
        live = keep & (torch.cumsum(stop.double(), 1) == 0)
        big = torch.full_like(rho, math.inf)
        m = torch.minimum(torch.where(valid[None], (rho / CUTOFF - 1).abs(), big),
                          torch.where(valid[None] & (rho <= CUTOFF), (a_raw / ALPHA_MIN - 1).abs(), big))
        m = torch.minimum(m, torch.where(keep, ((Tb * (1 - al)) / T_STOP - 1).abs(), big))
        # conditioning of the ray-disk intersection: FP32 loses about eps / sin(theta) of
        # (u, v), sin(theta) = |q2| / (|h_x| |h_y|); below 1e-3 the pixel counts as a margin pixel
        sin_t = q[..., 2].abs() / (hx.norm(dim=-1) * hy.norm(dim=-1))
        m = torch.minimum(m, torch.where(keep & (rho3 <= rho2), 0.1 * sin_t, big))
        # the depth switches between the intersection and the centre at rho3 = rho2
        m = torch.minimum(m, torch.where(keep, (rho3 / rho2 - 1).abs(), big))
        margin = m.min(1).values if m.shape[1] else torch.full_like(xs, math.inf)
    alpha = torch.where(live, torch.clamp(a_raw, max=ALPHA_MAX), torch.zeros_like(a_raw))
    Tb = torch.cumprod(torch.cat([torch.ones_like(alpha[:, :1]), 1 - alpha[:, :-1]], 1), 1)
    w = alpha * Tb
    zint = torch.where(live, zint, torch.zeros_like(zint))
    color = (w[..., None] * rgb[None]).sum(1)
    depth = (w * zint).sum(1)
    A = w.sum(1)
    normal = (w[..., None] * n[None]).sum(1)
    Ap = torch.cumsum(w, 1) - w
    Dp = torch.cumsum(w * zint, 1) - w * zint
    Ep = torch.cumsum(w * zint * zint, 1) - w * zint * zint
    dist = (w * (zint * zint * Ap - 2 * zint * Dp + Ep)).sum(1)
    return dict(color=color, depth=depth, alpha=A, normal=normal, distortion=dist,
                T=1 - A if A.numel() else A, ncontrib=live.sum(1)), margin


def _params(scene, grad: bool):
    P = {k: torch.tensor(np.asarray(getattr(scene, k), np.float64), requires_grad=grad)
         for k in ("means", "log_scales", "quats", "opacity_logits", "sh")}
    return P


def _run(scene, cameras, pixels, grad, chunk=4096):
    cams = scene.cameras if cameras is None else cameras
    P = _params(scene, grad)
    xis = [torch.zeros(6, dtype=torch.float64, requires_grad=grad) for _ in cams]
    views = []
    for vi, cam in enumerate(cams):
        S = _view(P, cam, xis[vi] if grad else None, scene.sh_degree)
        if pixels is None:
            ys, xs = np.mgrid[0:cam.H, 0:cam.W]
            lin = (ys * cam.W + xs).reshape(-1)
        else:
            lin = np.asarray(pixels[vi], np.int64)
        xs_all = torch.tensor((lin % cam.W).astype(np.float64))
        ys_all = torch.tensor((lin // cam.W).astype(np.float64))
        parts, margins = [], []
        for s in range(0, len(lin), chunk):
            o, mg = _composite(S, xs_all[s:s + chunk], ys_all[s:s + chunk])
            parts.append(o)
            margins.append(mg)
        out = {k: torch.cat([p[k] for p in parts]) if parts else torch.zeros(0) for k in parts[0]} if parts else {}
        out["margin"] = torch.cat(margins) if margins else torch.zeros(0)
        views.append((cam, out))
    return P, xis, views


def _shape(cam, a, full, channels=1):
    a = a.detach().numpy()
    if not full:
        return a.T if channels > 1 else a
    return a.T.reshape(channels, cam.H, cam.W) if channels > 1 else a.reshape(cam.H, cam.W)


def render_surfels(scene, pixels: Optional[List[np.ndarray]] = None, cameras=None):
    """Forward render of the surfel scene.  Returns per view dicts: color
    [3, H, W], depth, alpha, normal [3, H, W], distortion, T, ncontrib,
    margin (full images; pixel lists give [3, n] / [n])."""
    with torch.no_grad():
        _, _, views = _run(scene, cameras, pixels, grad=False)
    res = []
    full = pixels is None
    for cam, o in views:
        res.append(dict(color=_shape(cam, o["color"], full, 3), depth=_shape(cam, o["depth"], full),
                        alpha=_shape(cam, o["alpha"], full), normal=_shape(cam, o["normal"], full, 3),
                        distortion=_shape(cam, o["distortion"], full), T=_shape(cam, o["T"], full),
                        ncontrib=_shape(cam, o["ncontrib"].double(), full).astype(np.int64),
                        margin=_shape(cam, o["margin"], full)))
    return res


def render_surfels_backward(scene, gC, gD, gA, gN, gL, pixels: Optional[List[np.ndarray]] = None, cameras=None):
    """Forward + backward of sum(gC C + gD D + gA A + gN N + gL L) over the
    selected pixels (per view arrays shaped like the outputs).  Returns
    (per view forward dicts, grads dict of means, log_scales, quats,
    opacity_logits, sh, pose [V, 6])."""
    P, xis, views = _run(scene, cameras, pixels, grad=True)
    loss = torch.zeros((), dtype=torch.float64)
    res = []
    full = pixels is None
    for vi, (cam, o) in enumerate(views):
        f = lambda g, ch: torch.tensor(np.asarray(g, np.float64).reshape(ch, -1).T if ch > 1
                                       else np.asarray(g, np.float64).reshape(-1))
        loss = loss + (f(gC[vi], 3) * o["color"]).sum() + (f(gD[vi], 1) * o["depth"]).sum() + \
            (f(gA[vi], 1) * o["alpha"]).sum() + (f(gN[vi], 3) * o["normal"]).sum() + \
            (f(gL[vi], 1) * o["distortion"]).sum()
        res.append(dict(color=_shape(cam, o["color"], full, 3), depth=_shape(cam, o["depth"], full),
                        alpha=_shape(cam, o["alpha"], full), normal=_shape(cam, o["normal"], full, 3),
                        distortion=_shape(cam, o["distortion"], full), margin=_shape(cam, o["margin"], full)))
    loss.backward()
    g = {k: (P[k].grad.numpy() if P[k].grad is not None else np.zeros(P[k].shape)) for k in P}
    g["pose"] = np.stack([(x.grad.numpy() if x.grad is not None else np.zeros(6)) for x in xis])
    return res, g
