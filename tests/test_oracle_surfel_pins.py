"""Pins of the FP64 surfel (2DGS) oracle, oracle/surfel.py: closed forms, an
independent ray cast, a worked two-surfel case, central differences."""
import numpy as np
import pytest
import torch
from scipy.spatial.transform import Rotation

import oracle
from oracle import surfel as OS
from paper_2411_17660_b300 import scenes
from tests.test_oracle_pins import cam, dc_for_rgb, make_scene


def _quat(R):
    x, y, z, w = Rotation.from_matrix(R).as_quat()
    return np.array([w, x, y, z])


def test_sh_basis_matches_c_oracle():
    rng = np.random.default_rng(1)
    for _ in range(10):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        Y = OS.sh_basis_t(3, torch.tensor(d)).numpy()
        np.testing.assert_allclose(Y, oracle.sh_basis(3, d), atol=1e-15)


def test_fronto_parallel_disk_closed_form():
    """A disk facing the camera on the axis: rho3 = |x - c|^2 (z / (f s))^2."""
    c = cam(33, 41, 60.0)
    z, s, logit = 2.5, 0.05, 0.7
    rgb = np.array([0.3, 0.6, 0.9])
    sc = make_scene([[0.0], [0.0], [z]], np.log([[s], [s], [0.01]]), [[1.0], [0.0], [0.0], [0.0]],
                    [logit], dc_for_rgb(rgb)[:, None], 0, [c])
    out = OS.render_surfels(sc)[0]
    yy, xx = np.mgrid[0:33, 0:41]
    r2 = (xx - 20.5) ** 2 + (yy - 16.5) ** 2
    rho = np.minimum(r2 * (z / (60.0 * s)) ** 2, 2 * r2)
    sig = 1 / (1 + np.exp(-logit))
    a = sig * np.exp(-0.5 * rho)
    a = np.where((rho <= 9) & (a >= 1 / 255), np.minimum(a, 0.99), 0.0)
    np.testing.assert_allclose(out["alpha"], a, atol=1e-14)
    np.testing.assert_allclose(out["depth"], z * a, atol=1e-13)
    for k in range(3):
        np.testing.assert_allclose(out["color"][k], rgb[k] * a, atol=1e-14)
    np.testing.assert_allclose(out["normal"][2], -a, atol=1e-14)   # turned to face the camera
    assert not out["normal"][:2].any() and not out["distortion"].any()


def test_tilted_disk_matches_ray_cast():
    """alpha and depth of a tilted disk against an explicit ray-plane
    intersection solved with numpy (a different formulation)."""
    c = cam(30, 36, 50.0)
    R = Rotation.from_euler("xyz", [0.5, -0.4, 0.3]).as_matrix()
    mu, s = np.array([0.08, -0.05, 2.2]), np.array([0.09, 0.05, 0.01])
    sig = 0.8
    sc = make_scene(mu[:, None], np.log(s)[:, None], _quat(R)[:, None], [np.log(sig / (1 - sig))],
                    dc_for_rgb([0.5, 0.5, 0.5])[:, None], 0, [c])
    out = OS.render_surfels(sc)[0]
    K = np.array([[50.0, 0, c.cx], [0, 50.0, c.cy], [0, 0, 1]])
    uc = K @ mu
    uc = uc[:2] / uc[2]
    checked = 0
    for y in range(c.H):
        for x in range(c.W):
            d = np.linalg.solve(K, [x, y, 1.0])
            # mu + u s_u t_u + v s_v t_v = t d
            A = np.stack([s[0] * R[:, 0], s[1] * R[:, 1], -d], 1)
            u, v, _ = np.linalg.solve(A, -mu)
            rho = min(u * u + v * v, 2 * ((x - uc[0]) ** 2 + (y - uc[1]) ** 2))
            a = sig * np.exp(-0.5 * rho)
            a = min(a, 0.99) if (rho <= 9 and a >= 1 / 255) else 0.0
            zi = (mu + u * s[0] * R[:, 0] + v * s[1] * R[:, 1])[2]
            assert out["alpha"][y, x] == pytest.approx(a, abs=1e-12)
            assert out["depth"][y, x] == pytest.approx(a * zi, abs=1e-12)
            checked += a > 0
    assert checked > 20


def test_two_surfel_distortion_by_hand():
    c = cam(9, 9, 40.0)
    z1, z2 = 2.0, 2.6
    sc = make_scene([[0.0, 0.0], [0.0, 0.0], [z2, z1]], np.log([[0.2, 0.1], [0.2, 0.1], [0.01, 0.01]]),
                    [[1.0, 1.0], [0, 0], [0, 0], [0, 0]], [0.3, -0.2],
                    np.stack([dc_for_rgb([0.2] * 3), dc_for_rgb([0.8] * 3)], 1), 0, [c])
    o = OS.render_surfels(sc)[0]
    sig = lambda l: 1 / (1 + np.exp(-l))
    for (x, y) in [(4, 4), (5, 3), (6, 6)]:
        r2 = (x - 4.5) ** 2 + (y - 4.5) ** 2
        a1 = sig(-0.2) * np.exp(-0.5 * min(r2 * (z1 / (40 * 0.1)) ** 2, 2 * r2))
        a2 = sig(0.3) * np.exp(-0.5 * min(r2 * (z2 / (40 * 0.2)) ** 2, 2 * r2))
        w1, w2 = a1, a2 * (1 - a1)
        assert o["distortion"][y, x] == pytest.approx(w1 * w2 * (z1 - z2) ** 2, rel=1e-12)
        assert o["depth"][y, x] == pytest.approx(w1 * z1 + w2 * z2, rel=1e-12)


def _surfel_scene(seed, N=5, H=16, W=18, f=20.0, deg=1):
    rng = np.random.default_rng(seed)
    while True:
        means = np.stack([rng.uniform(-0.4, 0.4, N), rng.uniform(-0.3, 0.3, N), rng.uniform(1.6, 2.6, N)])
        q = rng.normal(size=(4, N))
        q[0] += 2.0   # mostly facing the camera
        ls = np.stack([rng.normal(-1.6, 0.2, N), rng.normal(-1.6, 0.2, N), np.full(N, -5.0)])
        K = (deg + 1) ** 2
        sh = rng.normal(0, 0.1, (3 * K, N))
        sh[:3] = rng.uniform(-1.2, 1.2, (3, N))
        sc = make_scene(means, ls, q, rng.uniform(-0.5, 1.5, N), sh, deg, [cam(H, W, f)])
        o = OS.render_surfels(sc)[0]
        if o["margin"].min() > 3e-3 and (o["ncontrib"] > 0).mean() > 0.3:
            return sc


def _surfel_loss(sc, w):
    o = OS.render_surfels(sc)[0]
    return sum((w[k] * o[k]).sum() for k in w)


def test_surfel_gradients_match_central_fd():
    sc = _surfel_scene(3)
    c = sc.cameras[0]
    rng = np.random.default_rng(4)
    w = dict(color=rng.uniform(-1, 1, (3, c.H, c.W)), depth=rng.uniform(-1, 1, (c.H, c.W)),
             alpha=rng.uniform(-1, 1, (c.H, c.W)), normal=rng.uniform(-1, 1, (3, c.H, c.W)),
             distortion=rng.uniform(-1, 1, (c.H, c.W)))
    _, g = OS.render_surfels_backward(sc, [w["color"]], [w["depth"]], [w["alpha"]], [w["normal"]],
                                      [w["distortion"]])
    h = 1e-6
    for name in ("means", "log_scales", "quats", "opacity_logits", "sh"):
        arr = getattr(sc, name)
        fd = np.zeros_like(arr)
        flat = arr.reshape(-1)
        for i in range(flat.size):
            keep = flat[i]
            flat[i] = keep + h
            lp = _surfel_loss(sc, w)
            flat[i] = keep - h
            lm = _surfel_loss(sc, w)
            flat[i] = keep
            fd.reshape(-1)[i] = (lp - lm) / (2 * h)
        err = np.linalg.norm(g[name] - fd) / max(np.linalg.norm(fd), 1e-30)
        assert err < 1e-6, (name, err)
    assert not g["log_scales"][2].any()   # the third scale of a flat disk is unused


def test_surfel_pose_gradient_matches_central_fd():
    sc = _surfel_scene(5)
    c = sc.cameras[0]
    rng = np.random.default_rng(6)
    w = dict(color=rng.uniform(-1, 1, (3, c.H, c.W)), depth=rng.uniform(-1, 1, (c.H, c.W)),
             alpha=np.zeros((c.H, c.W)), normal=rng.uniform(-1, 1, (3, c.H, c.W)),
             distortion=rng.uniform(-1, 1, (c.H, c.W)))
    _, g = OS.render_surfels_backward(sc, [w["color"]], [w["depth"]], [w["alpha"]], [w["normal"]],
                                      [w["distortion"]])
    from scipy.linalg import expm
    T = np.vstack([c.T_cw, [0, 0, 0, 1]])
    fd = np.zeros(6)
    h = 1e-6
    for k in range(6):
        vals = []
        for sgn in (1, -1):
            xi = np.zeros(6)
            xi[k] = sgn * h
            X = np.zeros((4, 4))
            X[:3, :3] = [[0, -xi[5], xi[4]], [xi[5], 0, -xi[3]], [-xi[4], xi[3], 0]]
            X[:3, 3] = xi[:3]
            Tp = expm(X) @ T
            cp = scenes.Camera(c.H, c.W, c.fx, c.fy, c.cx, c.cy, Tp[:3])
            vals.append(_surfel_loss(sc.with_cameras([cp]), w))
        fd[k] = (vals[0] - vals[1]) / (2 * h)
    np.testing.assert_allclose(g["pose"][0], fd, rtol=1e-6, atol=1e-9)
