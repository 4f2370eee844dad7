"""Seeded synthetic scenes for the Gaussian rasteriser.

This module only draws inputs: Gaussian parameters, cameras and loss targets.
It holds none of the rendering arithmetic, so the FP64 oracle and the CUDA path
can both consume it without sharing any of the method.

Stand-ins: the paper evaluates on TUM-RGBD, Replica and phone videos (Sec. 4,
"Datasets"), which are not available here.  The five workloads below reproduce
their shape instead: indoor rooms of Replica size (~120k-300k Gaussians,
Supp. Tab. "full render"), an 8-keyframe mapping window, an uneven 16-view
window and an outdoor 32-view window (the mapper batch of Supp. Sec. 1.2:
new keyframes + 10 last + 20 random).

Parameter conventions (all float32, planar "[K][N]" so that Gaussian g of
component k sits at k*N + g):
  means            [3][N]   world position P (Sec. 3.3)
  log_scales       [3][N]   log of the axis scales s
  quats            [4][N]   rotation r as an unnormalised quaternion (w, x, y, z)
  opacity_logits   [N]      density sigma before the sigmoid
  sh               [(d+1)^2 * 3][N]  SH coefficients, coefficient-major then
                            channel: row k*3 + c holds coefficient k of channel c
Cameras: pinhole (fx, fy, cx, cy), pixel centres at integer coordinates,
T_cw = [W | t] (row-major 3x4) maps world to camera, camera looks down +z.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional

import numpy as np
from scipy.spatial.transform import Rotation

# Half-width of the DC coefficient range.  With the real-SH constant
# Y00 = 1/(2 sqrt(pi)), DC coefficients uniform on [-sqrt(pi), sqrt(pi)]
# give a DC colour uniform on [0, 1] (the configs' "RGB uniform [0,1]").
SH_DC_HALF_RANGE = float(np.sqrt(np.pi))


@dataclasses.dataclass
class Camera:
    H: int
    W: int
    fx: float
    fy: float
    cx: float
    cy: float
    T_cw: np.ndarray  # float32 [3, 4] world -> camera


@dataclasses.dataclass
class Scene:
    name: str
    sh_degree: int
    means: np.ndarray
    log_scales: np.ndarray
    quats: np.ndarray
    opacity_logits: np.ndarray
    sh: np.ndarray
    cameras: List[Camera]
    target_color: List[np.ndarray]   # per view float32 [3, H, W]
    target_depth: List[np.ndarray]   # per view float32 [H, W]
    depth_weight: float              # weight of the L1 depth term in the loss

    @property
    def N(self) -> int:
        return int(self.means.shape[1])

    @property
    def V(self) -> int:
        return len(self.cameras)

    @property
    def pixels(self) -> int:
        return int(sum(c.H * c.W for c in self.cameras))

    def subset(self, idx: np.ndarray) -> "Scene":
        """The same scene restricted to Gaussians idx (in that order)."""
        return dataclasses.replace(
            self,
            means=np.ascontiguousarray(self.means[:, idx]),
            log_scales=np.ascontiguousarray(self.log_scales[:, idx]),
            quats=np.ascontiguousarray(self.quats[:, idx]),
            opacity_logits=np.ascontiguousarray(self.opacity_logits[idx]),
            sh=np.ascontiguousarray(self.sh[:, idx]),
        )

    def with_cameras(self, cams: List[Camera], colors=None, depths=None) -> "Scene":
        rng = np.random.default_rng(12345)
        if colors is None:
            colors = [rng.uniform(0, 1, (3, c.H, c.W)).astype(np.float32) for c in cams]
        if depths is None:
            depths = [rng.uniform(0.5, 6.0, (c.H, c.W)).astype(np.float32) for c in cams]
        return dataclasses.replace(self, cameras=list(cams), target_color=list(colors),
                                   target_depth=list(depths))


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


def random_quats(rng, N) -> np.ndarray:
    """Uniform on S^3: normalised 4-D normals, stored unnormalised-safe."""
    q = rng.standard_normal((4, N))
    q /= np.linalg.norm(q, axis=0, keepdims=True)
    return _f32(q)


def sh_coeffs(rng, N, degree) -> np.ndarray:
    """DC colour uniform on [0,1]; higher bands N(0, 0.05) raw coefficients."""
    K = (degree + 1) ** 2
    sh = np.empty((K * 3, N), dtype=np.float64)
    sh[0:3] = rng.uniform(-SH_DC_HALF_RANGE, SH_DC_HALF_RANGE, (3, N))
    if K > 1:
        sh[3:] = rng.normal(0.0, 0.05, (3 * (K - 1), N))
    return _f32(sh)


def distinct_f32(x: np.ndarray) -> bool:
    return np.unique(x.astype(np.float32)).size == x.size


def identity_pose() -> np.ndarray:
    return _f32(np.hstack([np.eye(3), np.zeros((3, 1))]))


def pose_from_c2w(R_wc: np.ndarray, C: np.ndarray) -> np.ndarray:
    """World->camera [W | t] from a camera-to-world rotation and centre."""
    W = R_wc.T
    return _f32(np.hstack([W, (-W @ C).reshape(3, 1)]))


def trajectory(rng, V, step_m=0.1, step_deg=5.0, max_off_axis_deg=45.0,
               start=(0.0, 0.0, 0.0)) -> List[np.ndarray]:
    """Smooth random camera path: each keyframe moves step_m in a random
    direction and turns step_deg about a random axis, keeping the viewing
    direction within max_off_axis_deg of world +z (looking into the scene)."""
    R = np.eye(3)
    C = np.asarray(start, dtype=np.float64)
    poses = [pose_from_c2w(R, C)]
    cos_max = np.cos(np.deg2rad(max_off_axis_deg))
    while len(poses) < V:
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        a = rng.standard_normal(3)
        a /= np.linalg.norm(a)
        R_new = Rotation.from_rotvec(np.deg2rad(step_deg) * a).as_matrix() @ R
        if R_new[2, 2] < cos_max:   # camera +z in world = third column of R
            continue
        R, C = R_new, C + step_m * d
        poses.append(pose_from_c2w(R, C))
    return poses


def room_points(rng, N, size=(6.0, 3.0, 4.0), wall_frac=0.7, wall_depth=0.05):
    """Room of size (x, y vertical, z) centred at the origin: wall_frac of the
    points lie within wall_depth inside a wall (face chosen by area), the rest
    uniform in the volume."""
    hx, hy, hz = (s / 2 for s in size)
    n_wall = int(round(N * wall_frac))
    pts = np.empty((N, 3))
    # faces: +-x (area y*z), +-y (x*z), +-z (x*y)
    areas = np.array([size[1] * size[2]] * 2 + [size[0] * size[2]] * 2 + [size[0] * size[1]] * 2)
    face = rng.choice(6, size=n_wall, p=areas / areas.sum())
    u = rng.uniform(-1, 1, (n_wall, 3)) * np.array([hx, hy, hz])
    depth = rng.uniform(0, wall_depth, n_wall)
    axis = face // 2
    sign = np.where(face % 2 == 0, 1.0, -1.0)
    half = np.array([hx, hy, hz])[axis]
    u[np.arange(n_wall), axis] = sign * (half - depth)
    pts[:n_wall] = u
    pts[n_wall:] = rng.uniform(-1, 1, (N - n_wall, 3)) * np.array([hx, hy, hz])
    return pts[rng.permutation(N)]


def _scene(name, degree, means_xyz, log_scales, rng, logit_sigma, cams, depth_weight):
    N = means_xyz.shape[0]
    scene = Scene(
        name=name, sh_degree=degree,
        means=_f32(means_xyz.T), log_scales=_f32(log_scales),
        quats=random_quats(rng, N),
        opacity_logits=_f32(rng.normal(0.0, logit_sigma, N)),
        sh=sh_coeffs(rng, N, degree), cameras=[], target_color=[], target_depth=[],
        depth_weight=depth_weight)
    tgt = np.random.default_rng(rng.integers(1 << 62))
    colors = [_f32(tgt.uniform(0, 1, (3, c.H, c.W))) for c in cams]
    depths = [_f32(tgt.uniform(0.5, 6.0, (c.H, c.W))) for c in cams]
    return scene.with_cameras(cams, colors, depths)


def config_small(seed=0, N=2000, H=120, W=160, f=150.0) -> Scene:
    """Single 160x120 view, 2,000 Gaussians in a camera-frame box, SH degree 0."""
    rng = np.random.default_rng(seed)
    while True:
        xyz = np.stack([rng.uniform(-1, 1, N), rng.uniform(-1, 1, N), rng.uniform(2, 6, N)], 1)
        if distinct_f32(xyz[:, 2]):
            break
    ls = rng.normal(-3.0, 0.5, (3, N))
    cam = Camera(H, W, f, f, W / 2, H / 2, identity_pose())
    return _scene("small-160x120-2k-deg0", 0, xyz, ls, rng, 1.0, [cam], 0.0)


def config_room(seed=1, N=300_000, H=680, W=1200, f=600.0) -> Scene:
    """Single 1200x680 view from the centre of a 6x3x4 m room, 300k Gaussians, SH degree 3."""
    rng = np.random.default_rng(seed)
    xyz = room_points(rng, N)
    ls = rng.normal(-4.0, 0.7, (3, N))
    cam = Camera(H, W, f, f, W / 2, H / 2, identity_pose())
    return _scene(f"room-{W}x{H}-{N // 1000}k-deg3", 3, xyz, ls, rng, 1.5, [cam], 0.1)


def config_window(seed=2, N=100_000, V=8, H=480, W=640, f=500.0) -> Scene:
    """8-keyframe mapping window of 640x480 views on a smooth path in the room, 100k Gaussians."""
    rng = np.random.default_rng(seed)
    xyz = room_points(rng, N)
    ls = rng.normal(-4.0, 0.7, (3, N))
    cams = [Camera(H, W, f, f, W / 2, H / 2, T) for T in trajectory(rng, V)]
    return _scene(f"window-{V}x{W}x{H}-{N // 1000}k-deg3", 3, xyz, ls, rng, 1.5, cams, 0.1)


def config_uneven(seed=3, N=800_000, V=16, res_scale=1.0) -> Scene:
    """16 keyframes at resolutions drawn from {320x240, 640x480, 1200x680};
    half of the 800k Gaussians in two 1 m balls with small scales."""
    rng = np.random.default_rng(seed)
    n_ball = N // 2
    centres = np.array([[-1.0, 0.2, 1.2], [0.9, -0.2, 1.6]])
    which = rng.integers(0, 2, n_ball)
    d = rng.standard_normal((n_ball, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    r = 0.5 * rng.uniform(0, 1, n_ball) ** (1.0 / 3.0)
    ball = centres[which] + d * r[:, None]
    room = room_points(rng, N - n_ball)
    xyz = np.concatenate([ball, room])
    ls = np.concatenate([rng.normal(-5.0, 0.5, (3, n_ball)), rng.normal(-4.0, 0.7, (3, N - n_ball))], 1)
    perm = rng.permutation(N)
    xyz, ls = xyz[perm], ls[:, perm]
    res = [(240, 320), (480, 640), (680, 1200)]
    picks = rng.integers(0, 3, V)
    cams = []
    for T, p in zip(trajectory(rng, V), picks):
        H, W = res[p]
        H, W = max(8, int(round(H * res_scale))), max(8, int(round(W * res_scale)))
        f = 500.0 * W / 640.0
        cams.append(Camera(H, W, f, f, W / 2, H / 2, T))
    return _scene(f"uneven-{V}views-{N // 1000}k-deg3", 3, xyz, ls, rng, 1.5, cams, 0.1)


def config_outdoor(seed=4, N=2_000_000, V=32, H=1080, W=1920, f=1400.0) -> Scene:
    """32 keyframes of 1920x1080 over an outdoor-like scene of 2M Gaussians:
    60% within 0.1 m of a ground plane y=+1.5, 40% in a 40x11.5x39 m box,
    heavy-tailed scales clipped at 0.5 m."""
    rng = np.random.default_rng(seed)
    n_g = int(round(0.6 * N))
    ground = np.stack([rng.uniform(-20, 20, n_g), 1.5 + rng.uniform(-0.1, 0.1, n_g),
                       rng.uniform(1, 40, n_g)], 1)
    free = np.stack([rng.uniform(-20, 20, N - n_g), rng.uniform(-10, 1.5, N - n_g),
                     rng.uniform(1, 40, N - n_g)], 1)
    xyz = np.concatenate([ground, free])[rng.permutation(N)]
    ls = np.minimum(rng.normal(-4.0, 1.2, (3, N)), np.log(0.5))
    cams = [Camera(H, W, f, f, W / 2, H / 2, T) for T in trajectory(rng, V)]
    return _scene(f"outdoor-{V}x{W}x{H}-{N // 1000}k-deg3", 3, xyz, ls, rng, 2.0, cams, 0.1)


CONFIGS = {
    "small": config_small,
    "room": config_room,
    "window": config_window,
    "uneven": config_uneven,
    "outdoor": config_outdoor,
}


def make(name: str, **kw) -> Scene:
    return CONFIGS[name](**kw)


def sparse_pixel_grads(scene: Scene, per_view: int, seed: int = 7):
    """Upstream gradients that are zero except on `per_view` random pixels of
    each view.  Used to check full-size gradients against the oracle, which
    then only needs those pixels.  Returns (pixels, gC, gD, gA) lists."""
    rng = np.random.default_rng(seed)
    pix, gC, gD, gA = [], [], [], []
    for c in scene.cameras:
        idx = rng.choice(c.H * c.W, size=min(per_view, c.H * c.W), replace=False)
        idx.sort()
        pix.append(idx.astype(np.int64))
        gC.append(_f32(rng.uniform(-1, 1, (3, idx.size))))
        gD.append(_f32(rng.uniform(-1, 1, idx.size)))
        gA.append(_f32(rng.uniform(-1, 1, idx.size)))
    return pix, gC, gD, gA
