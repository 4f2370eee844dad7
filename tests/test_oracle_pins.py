"""Pins of the FP64 oracle against facts that do not come from the oracle.

Each test below checks the oracle against something fixed by the paper or by
mathematics: a closed-form footprint, a hand-composited worked case,
quadrature and the SH addition theorem, a library rotation, a finite-
difference Jacobian of the pinhole model, brute force, invariants,
symmetries and central finite differences of the oracle's own forward.
"""
import numpy as np
import pytest
from numpy.polynomial import legendre
from scipy.spatial.transform import Rotation

import oracle
from paper_2411_17660_b300 import scenes

Y00 = 1.0 / (2.0 * np.sqrt(np.pi))  # textbook real SH constant


def make_scene(means, log_scales, quats, logits, sh, deg, cams):
    return scenes.Scene(
        name="pin", sh_degree=deg,
        means=np.asarray(means, np.float64), log_scales=np.asarray(log_scales, np.float64),
        quats=np.asarray(quats, np.float64), opacity_logits=np.asarray(logits, np.float64),
        sh=np.asarray(sh, np.float64), cameras=list(cams), target_color=[], target_depth=[],
        depth_weight=0.0)


def cam(H, W, f, T=None, cx=None, cy=None):
    T = np.hstack([np.eye(3), np.zeros((3, 1))]) if T is None else np.asarray(T, np.float64)
    return scenes.Camera(H, W, f, f, W / 2 if cx is None else cx, H / 2 if cy is None else cy, T)


def dc_for_rgb(rgb):
    """SH degree-0 coefficients giving colour rgb (c = Y00 * sh + 0.5)."""
    return (np.asarray(rgb, np.float64) - 0.5) / Y00


# ---------------------------------------------------------------- SH basis

def test_sh_orthonormal_by_quadrature():
    # Gauss-Legendre in cos(theta) x uniform phi: exact for the degree <= 6 products
    xs, ws = legendre.leggauss(16)
    phis = np.arange(32) * 2 * np.pi / 32
    M = np.zeros((16, 16))
    for x, w in zip(xs, ws):
        s = np.sqrt(1 - x * x)
        for p in phis:
            Y = oracle.sh_basis(3, [s * np.cos(p), s * np.sin(p), x])
            M += w * (2 * np.pi / 32) * np.outer(Y, Y)
    np.testing.assert_allclose(M, np.eye(16), atol=1e-12)


def test_sh_addition_theorem():
    # sum_m Y_lm(a) Y_lm(b) = (2l+1)/(4 pi) P_l(a.b), independent of the sign convention
    rng = np.random.default_rng(0)
    for _ in range(20):
        a, b = rng.standard_normal(3), rng.standard_normal(3)
        a /= np.linalg.norm(a)
        b /= np.linalg.norm(b)
        Ya, Yb = oracle.sh_basis(3, a), oracle.sh_basis(3, b)
        for l in range(4):
            band = slice(l * l, (l + 1) * (l + 1))
            Pl = legendre.legval(a @ b, [0] * l + [1])
            assert abs(Ya[band] @ Yb[band] - (2 * l + 1) / (4 * np.pi) * Pl) < 1e-13


def test_sh_degree_truncation_and_phase():
    d = np.array([0.3, -0.5, 0.8]); d /= np.linalg.norm(d)
    Y0, Y3 = oracle.sh_basis(0, d), oracle.sh_basis(3, d)
    assert Y0[0] == pytest.approx(Y00) and np.all(Y0[1:] == 0)
    # Condon-Shortley phase: Y_1,-1 = -k y, Y_1,0 = k z, Y_1,1 = -k x
    k = np.sqrt(3 / (4 * np.pi))
    np.testing.assert_allclose(Y3[1:4], [-k * d[1], k * d[2], -k * d[0]], rtol=1e-14)


# ---------------------------------------------------------------- rotations

def test_quat_to_rot_matches_scipy():
    rng = np.random.default_rng(1)
    for _ in range(50):
        q = rng.standard_normal(4) * rng.uniform(0.1, 3)
        R = oracle.quat_to_rot(q)
        ref = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()  # scipy is (x,y,z,w)
        np.testing.assert_allclose(R, ref, atol=1e-14)


# ---------------------------------------------------------------- projection

def test_projected_covariance_matches_fd_jacobian():
    """Sigma' equals J W Sigma W^T J^T + 0.3 I with J the numerical Jacobian of
    the pinhole model, Sigma from scipy's rotation; u, v the pinhole image."""
    rng = np.random.default_rng(2)
    Rwc = Rotation.from_rotvec([0.1, -0.2, 0.05]).as_matrix()
    C = np.array([0.3, -0.1, -0.5])
    T = np.hstack([Rwc.T, (-Rwc.T @ C)[:, None]])
    c = cam(60, 80, 70.0, T, cx=41.5, cy=29.0)
    N = 12
    mu = np.stack([rng.uniform(-0.8, 0.8, N), rng.uniform(-0.6, 0.6, N), rng.uniform(2, 5, N)])
    ls = rng.normal(-2.5, 0.4, (3, N))
    q = rng.standard_normal((4, N))
    sc = make_scene(mu, ls, q, rng.normal(0, 1, N), np.zeros((3, N)), 0, [c])
    P = oracle.project(sc, 0)
    W, t = T[:, :3], T[:, 3]

    def pi(p):
        return np.array([c.fx * p[0] / p[2] + c.cx, c.fy * p[1] / p[2] + c.cy])

    for g in range(N):
        pc = W @ mu[:, g] + t
        assert P["valid"][g] == 1
        np.testing.assert_allclose([P["u"][g], P["v"][g]], pi(pc), rtol=1e-14)
        assert P["z"][g] == pytest.approx(pc[2], rel=1e-14)
        J = np.zeros((2, 3))
        for k in range(3):
            h = 1e-5 * pc[2]
            e = np.zeros(3); e[k] = h
            J[:, k] = (pi(pc + e) - pi(pc - e)) / (2 * h)
        R = Rotation.from_quat([q[1, g], q[2, g], q[3, g], q[0, g]]).as_matrix()
        Sig = R @ np.diag(np.exp(2 * ls[:, g])) @ R.T
        S2 = J @ W @ Sig @ W.T @ J.T + 0.3 * np.eye(2)
        np.testing.assert_allclose([P["cov0"][g], P["cov1"][g], P["cov2"][g]],
                                   [S2[0, 0], S2[0, 1], S2[1, 1]], rtol=1e-8, atol=1e-9)
        Ci = np.linalg.inv(S2)
        np.testing.assert_allclose([P["conic0"][g], P["conic1"][g], P["conic2"][g]],
                                   [Ci[0, 0], Ci[0, 1], Ci[1, 1]], rtol=1e-7, atol=1e-9)


def test_near_plane_cull():
    c = cam(20, 20, 20.0)
    mu = np.array([[0.0, 0.0], [0.0, 0.0], [0.19, 0.21]])
    sc = make_scene(mu, np.full((3, 2), -3.0), np.array([[1.0, 1.0], [0, 0], [0, 0], [0, 0]]),
                    np.zeros(2), np.zeros((3, 2)), 0, [c])
    P = oracle.project(sc, 0)
    assert list(P["valid"]) == [0, 1]


# ---------------------------------------------------------------- compositing

def _iso_alpha(o, f, s, z, r2):
    """Closed-form alpha of an isotropic Gaussian on the optical axis."""
    var = (f * s / z) ** 2 + 0.3
    d2 = r2 / var
    a = o * np.exp(-0.5 * d2)
    return np.where((d2 <= 9) & (a >= 1 / 255), np.minimum(a, 0.99), 0.0)


def test_single_isotropic_gaussian_closed_form():
    c = cam(48, 64, 100.0)
    z, s, logit = 4.0, 0.05, 1.5
    rgb = np.array([0.2, 0.5, 0.9])
    sc = make_scene([[0.0], [0.0], [z]], np.full((3, 1), np.log(s)), [[0.3], [0.5], [-0.2], [0.7]],
                    [logit], dc_for_rgb(rgb)[:, None], 0, [c])
    out = oracle.render(sc)[0]
    yy, xx = np.mgrid[0:48, 0:64]
    r2 = (xx - 32.0) ** 2 + (yy - 24.0) ** 2
    a = _iso_alpha(1 / (1 + np.exp(-logit)), 100.0, s, z, r2)
    np.testing.assert_allclose(out["alpha"], a, atol=1e-13)
    np.testing.assert_allclose(out["T"], 1 - a, atol=1e-13)
    np.testing.assert_allclose(out["depth"], z * a, atol=1e-12)
    for k in range(3):
        np.testing.assert_allclose(out["color"][k], rgb[k] * a, atol=1e-13)
    assert out["ncontrib"].max() == 1 and out["ncontrib"].sum() == (a > 0).sum()


def test_two_gaussian_worked_case():
    c = cam(9, 9, 50.0)
    z1, z2 = 2.0, 3.0
    s1, s2 = 0.04, 0.08
    l1, l2 = 0.4, 1.2
    c1, c2 = np.array([0.9, 0.1, 0.3]), np.array([0.2, 0.8, 0.6])
    sc = make_scene([[0.0, 0.0], [0.0, 0.0], [z2, z1]], np.log([[s2, s1]] * 3),
                    [[1.0, 1.0], [0, 0], [0, 0], [0, 0]], [l2, l1],
                    np.stack([dc_for_rgb(c2), dc_for_rgb(c1)], 1), 0, [c])
    out = oracle.render(sc)[0]
    sig = lambda l: 1 / (1 + np.exp(-l))
    for (x, y) in [(4, 4), (5, 4), (6, 6), (4, 7)]:
        r2 = (x - 4.5) ** 2 + (y - 4.5) ** 2
        a1 = float(_iso_alpha(sig(l1), 50.0, s1, z1, r2))
        a2 = float(_iso_alpha(sig(l2), 50.0, s2, z2, r2))
        np.testing.assert_allclose(out["color"][:, y, x], c1 * a1 + c2 * a2 * (1 - a1), atol=1e-13)
        assert out["depth"][y, x] == pytest.approx(z1 * a1 + z2 * a2 * (1 - a1), abs=1e-13)
        assert out["alpha"][y, x] == pytest.approx(a1 + a2 * (1 - a1), abs=1e-13)


def test_skip_and_stop_rules():
    """Front to back: a faint Gaussian (alpha < 1/255, skipped), alpha 0.9,
    alpha 0.99 (clamped), alpha 0.99 whose T would fall below 1e-4: stop."""
    c = cam(3, 3, 10.0, cx=1.0, cy=1.0)
    logit_of = lambda a: np.log(a / (1 - a))
    zs = [1.0, 2.0, 3.0, 4.0]
    alphas = [0.003, 0.9, 0.999, 0.999]
    rgbs = [np.array([1.0, 1.0, 1.0]), np.array([0.5, 0.0, 0.0]), np.array([0.0, 0.5, 0.0]),
            np.array([0.0, 0.0, 0.5])]
    N = 4
    mu = np.stack([np.zeros(N), np.zeros(N), zs])
    # large isotropic scale: G ~ 1 at the centre pixel (d2 = 0 exactly there)
    sc = make_scene(mu, np.full((3, N), 0.0), np.tile([[1.0], [0], [0], [0]], N),
                    [logit_of(a) for a in alphas], np.stack([dc_for_rgb(r) for r in rgbs], 1), 0, [c])
    out = oracle.render(sc, pixels=[np.array([4])])[0]  # pixel (1,1) = principal point
    assert out["ncontrib"][0] == 2
    expect = rgbs[1] * 0.9 + rgbs[2] * 0.99 * 0.1
    np.testing.assert_allclose(out["color"][:, 0], expect, atol=1e-14)
    assert out["T"][0] == pytest.approx(0.1 * 0.01, rel=1e-12)
    assert out["alpha"][0] + out["T"][0] == pytest.approx(1.0, abs=1e-14)


def _random_scene(rng, N, H, W, f, deg, pose=True, logit_hi=2.0):
    Tm = np.hstack([np.eye(3), np.zeros((3, 1))])
    if pose:
        Rwc = Rotation.from_rotvec(rng.normal(0, 0.05, 3)).as_matrix()
        C = rng.normal(0, 0.05, 3)
        Tm = np.hstack([Rwc.T, (-Rwc.T @ C)[:, None]])
    z = rng.uniform(2, 4, N)
    mu = np.stack([rng.uniform(-0.35, 0.35, N) * z * W / f, rng.uniform(-0.35, 0.35, N) * z * H / f, z])
    ls = rng.normal(np.log(2.0 * 3.0 / f), 0.3, (3, N))
    K = (deg + 1) ** 2
    sh = np.zeros((3 * K, N))
    sh[0:3] = dc_for_rgb(rng.uniform(0.2, 0.8, (3, N)))
    sh[3:] = rng.normal(0, 0.05, (3 * K - 3, N))
    logits = rng.uniform(-1.5, logit_hi, N)
    return make_scene(mu, ls, rng.standard_normal((4, N)), logits, sh, deg, [cam(H, W, f, Tm)])


def test_weights_sum_invariant():
    rng = np.random.default_rng(3)
    sc = _random_scene(rng, 40, 30, 40, 40.0, 3, logit_hi=4.0)
    out = oracle.render(sc)[0]
    np.testing.assert_allclose(out["alpha"] + out["T"], 1.0, atol=1e-12)
    assert (out["ncontrib"] > 0).mean() > 0.3


def test_bucketed_equals_brute_force():
    rng = np.random.default_rng(4)
    for trial in range(5):
        sc = _random_scene(rng, 50, 24, 32, 30.0, 3 if trial % 2 else 0)
        a = oracle.render(sc, brute=False)[0]
        b = oracle.render(sc, brute=True)[0]
        for k in ("color", "depth", "alpha", "T", "ncontrib"):
            np.testing.assert_array_equal(a[k], b[k])


def test_permutation_invariance():
    rng = np.random.default_rng(5)
    sc = _random_scene(rng, 60, 32, 40, 40.0, 3)
    perm = rng.permutation(60)
    a = oracle.render(sc)[0]
    b = oracle.render(sc.subset(perm))[0]
    for k in ("color", "depth", "alpha", "T"):
        np.testing.assert_array_equal(a[k], b[k])


def test_rigid_transform_invariance_degree0():
    """Moving the whole scene by a rigid motion and the camera with it leaves
    the image unchanged (SH degree 0: colour has no view dependence)."""
    rng = np.random.default_rng(6)
    sc = _random_scene(rng, 40, 30, 40, 40.0, 0)
    Q = Rotation.from_rotvec([0.4, -0.3, 0.8])
    s = np.array([1.0, -2.0, 0.5])
    q = sc.quats / np.linalg.norm(sc.quats, axis=0)
    rq = (Q * Rotation.from_quat(np.stack([q[1], q[2], q[3], q[0]], 1))).as_quat()
    q2 = np.stack([rq[:, 3], rq[:, 0], rq[:, 1], rq[:, 2]])
    mu2 = Q.as_matrix() @ sc.means + s[:, None]
    T = sc.cameras[0].T_cw
    W2 = T[:, :3] @ Q.as_matrix().T
    t2 = T[:, 3] - W2 @ s
    c2 = scenes.Camera(30, 40, 40.0, 40.0, 20.0, 15.0, np.hstack([W2, t2[:, None]]))
    sc2 = make_scene(mu2, sc.log_scales, q2, sc.opacity_logits, sc.sh, 0, [c2])
    a, b = oracle.render(sc)[0], oracle.render(sc2)[0]
    for k in ("color", "depth", "alpha"):
        np.testing.assert_allclose(a[k], b[k], atol=1e-10)


# ---------------------------------------------------------------- gradients

def _fd_scene(seed, deg=3, N=6):
    """Small scene whose every threshold decision has a relative margin > 2e-3
    and no alpha or colour clamp, so central differences straddle no kink."""
    rng = np.random.default_rng(seed)
    while True:
        sc = _random_scene(rng, N, 20, 24, 24.0, deg, logit_hi=2.0)
        out = oracle.render(sc)[0]
        P = oracle.project(sc, 0)
        if min(out["margin"].min(), out["zmargin"].min()) > 2e-3 and (out["ncontrib"] > 0).mean() > 0.2 and \
                min(P["r"].min(), P["g"].min(), P["b"].min()) > 0.05:
            return sc


def _loss(sc, wC, wD, wA):
    o = oracle.render(sc)[0]
    return (wC * o["color"]).sum() + (wD * o["depth"]).sum() + (wA * o["alpha"]).sum()


def _upstream(sc, seed):
    rng = np.random.default_rng(seed)
    c = sc.cameras[0]
    return rng.uniform(-1, 1, (3, c.H, c.W)), rng.uniform(-1, 1, (c.H, c.W)), rng.uniform(-1, 1, (c.H, c.W))


@pytest.mark.parametrize("seed", [10, 11])
def test_param_gradients_match_central_fd(seed):
    sc = _fd_scene(seed)
    wC, wD, wA = _upstream(sc, seed)
    _, g = oracle.render_backward(sc, [wC], [wD], [wA])
    h = 1e-6
    for name in ("means", "log_scales", "quats", "opacity_logits", "sh"):
        arr = getattr(sc, name)
        fd = np.zeros_like(arr, dtype=np.float64)
        flat = arr.reshape(-1)
        for i in range(flat.size):
            keep = flat[i]
            flat[i] = keep + h
            lp = _loss(sc, wC, wD, wA)
            flat[i] = keep - h
            lm = _loss(sc, wC, wD, wA)
            flat[i] = keep
            fd.reshape(-1)[i] = (lp - lm) / (2 * h)
        an = g[name]
        err = np.linalg.norm(an - fd) / max(np.linalg.norm(fd), 1e-30)
        assert err < 1e-6, (name, err)


def _pose_fd(sc, wC, wD, wA, h=1e-6):
    c = sc.cameras[0]
    T = np.vstack([c.T_cw, [0, 0, 0, 1]])
    fd = np.zeros(6)
    for k in range(6):
        vals = []
        for sgn in (1, -1):
            xi = np.zeros(6); xi[k] = sgn * h
            E = np.eye(4)
            E[:3, :3] = Rotation.from_rotvec(xi[3:]).as_matrix()
            E[:3, 3] = xi[:3]
            T2 = (E @ T)[:3]
            c2 = scenes.Camera(c.H, c.W, c.fx, c.fy, c.cx, c.cy, T2)
            vals.append(_loss(sc.with_cameras([c2], [None], [None]), wC, wD, wA))
        fd[k] = (vals[0] - vals[1]) / (2 * h)
    return fd


@pytest.mark.parametrize("seed", [20, 21])
def test_pose_gradient_matches_central_fd(seed):
    sc = _fd_scene(seed)
    wC, wD, wA = _upstream(sc, seed)
    _, g = oracle.render_backward(sc, [wC], [wD], [wA])
    fd = _pose_fd(sc, wC, wD, wA)
    np.testing.assert_allclose(g["pose"][0], fd, rtol=2e-6, atol=1e-7 * np.abs(fd).max())


# ------------------------------------------------ clamped branches (3DGS conventions)

def _fd_all(sc, wC, wD, wA, h=1e-6):
    """Central differences of L = <wC, C> + <wD, D> + <wA, A> for every
    parameter class and the six pose dofs of view 0."""
    fd = {}
    for name in ("means", "log_scales", "quats", "opacity_logits", "sh"):
        arr = getattr(sc, name)
        out = np.zeros_like(arr, dtype=np.float64)
        flat = arr.reshape(-1)
        for i in range(flat.size):
            keep = flat[i]
            flat[i] = keep + h
            lp = _loss(sc, wC, wD, wA)
            flat[i] = keep - h
            lm = _loss(sc, wC, wD, wA)
            flat[i] = keep
            out.reshape(-1)[i] = (lp - lm) / (2 * h)
        fd[name] = out
    fd["pose"] = _pose_fd(sc, wC, wD, wA, h)
    return fd


def _assert_matches_fd(g, fd, tol=1e-6):
    for name, ref in fd.items():
        an = g[name][0] if name == "pose" else g[name]
        err = np.linalg.norm(an - ref) / max(np.linalg.norm(ref), 1e-30)
        assert err < tol, (name, err)


def test_projection_beyond_the_jacobian_clamp():
    """Beyond 1.3 x the half field of view the EWA Jacobian is taken at the
    clamped direction: Sigma' = J W Sigma W^T J^T + 0.3 I with J the numerical
    Jacobian of the pinhole model at (clip(x/z) z, clip(y/z) z, z), each ratio
    clipped to +-1.3 (W/2)/fx, +-1.3 (H/2)/fy; the pixel mean (u, v) is the
    unclamped pinhole image.  Points just inside the limit are not clamped."""
    c = cam(40, 64, 50.0, cx=31.0, cy=20.5)
    limx, limy = 1.3 * 32 / 50.0, 1.3 * 20 / 50.0
    ratios = [(0.95, 0.0), (1.05, 0.0), (1.6, 0.2), (-1.3, 0.5), (0.3, 1.04), (-0.2, -2.0), (1.2, -1.4),
              (-0.97, 0.99)]
    N = len(ratios)
    z = np.linspace(2.0, 5.0, N)
    mu = np.stack([[rx * limx * zz for (rx, _), zz in zip(ratios, z)],
                   [ry * limy * zz for (_, ry), zz in zip(ratios, z)], z])
    rng = np.random.default_rng(7)
    ls = rng.normal(-2.0, 0.3, (3, N))
    q = rng.standard_normal((4, N))
    sc = make_scene(mu, ls, q, np.zeros(N), np.zeros((3, N)), 0, [c])
    P = oracle.project(sc, 0)

    def pi(p):
        return np.array([c.fx * p[0] / p[2] + c.cx, c.fy * p[1] / p[2] + c.cy])

    for g, (rx, ry) in enumerate(ratios):
        pc = mu[:, g]
        assert P["clamp_x"][g] == (abs(rx) > 1) and P["clamp_y"][g] == (abs(ry) > 1)
        np.testing.assert_allclose([P["u"][g], P["v"][g]], pi(pc), rtol=1e-14)
        pt = np.array([np.clip(pc[0] / pc[2], -limx, limx) * pc[2], np.clip(pc[1] / pc[2], -limy, limy) * pc[2], pc[2]])
        J = np.zeros((2, 3))
        for k in range(3):
            e = np.zeros(3); e[k] = 1e-5 * pc[2]
            J[:, k] = (pi(pt + e) - pi(pt - e)) / (2e-5 * pc[2])
        R = Rotation.from_quat([q[1, g], q[2, g], q[3, g], q[0, g]]).as_matrix()
        S2 = J @ R @ np.diag(np.exp(2 * ls[:, g])) @ R.T @ J.T + 0.3 * np.eye(2)
        np.testing.assert_allclose([P["cov0"][g], P["cov1"][g], P["cov2"][g]],
                                   [S2[0, 0], S2[0, 1], S2[1, 1]], rtol=1e-8, atol=1e-9)


def _clamped_jacobian_scene(seed):
    """Gaussians whose means lie beyond the Jacobian clamp (x/z or y/z past
    1.3 x the half field of view, by more than 5 %) with footprints that
    still cover pixels, plus two on-screen ones; every threshold decision has
    a margin > 2e-3 and every colour is above 0.05."""
    rng = np.random.default_rng(seed)
    H, W, f = 20, 24, 24.0
    limx, limy = 1.3 * (W / 2) / f, 1.3 * (H / 2) / f
    while True:
        N = 6
        z = rng.uniform(2, 3.5, N)
        rx = np.concatenate([rng.choice([-1, 1], 3) * rng.uniform(1.08, 1.3, 3), rng.uniform(-0.5, 0.5, 3)])
        ry = np.concatenate([rng.uniform(-0.5, 0.5, 3), rng.choice([-1, 1], 1) * rng.uniform(1.08, 1.3, 1),
                             rng.uniform(-0.5, 0.5, 2)])
        ry[0] = rng.choice([-1, 1]) * rng.uniform(1.08, 1.25)      # one clamped in both ratios
        mu = np.stack([rx * limx * z, ry * limy * z, z])
        ls = np.log(rng.uniform(3.5, 5.0, (3, N)) * z / f)         # ~4 px footprints
        ls[:, 4:] = np.log(rng.uniform(1.5, 2.5, (3, 2)) * z[4:] / f)
        sh = np.zeros((48, N))
        sh[0:3] = dc_for_rgb(rng.uniform(0.2, 0.8, (3, N)))
        sh[3:] = rng.normal(0, 0.05, (45, N))
        Rwc = Rotation.from_rotvec(rng.normal(0, 0.02, 3)).as_matrix()
        Tm = np.hstack([Rwc.T, np.zeros((3, 1))])
        sc = make_scene(Rwc @ mu, ls, rng.standard_normal((4, N)), rng.uniform(-0.5, 1.5, N), sh, 3,
                        [cam(H, W, f, Tm)])
        out = oracle.render(sc)[0]
        P = oracle.project(sc, 0)
        pc = Rwc.T @ sc.means
        ratio = np.maximum(np.abs(pc[0] / pc[2]) / limx, np.abs(pc[1] / pc[2]) / limy)
        if min(out["margin"].min(), out["zmargin"].min()) > 2e-3 and \
                np.all(np.abs(np.abs(pc[0] / pc[2]) / limx - 1) > 1e-2) and \
                np.all(np.abs(np.abs(pc[1] / pc[2]) / limy - 1) > 1e-2) and \
                min(P["r"].min(), P["g"].min(), P["b"].min()) > 0.05 and \
                (P["clamp_x"] + P["clamp_y"] > 0).sum() >= 3 and (ratio > 1).sum() >= 3:
            return sc, P


@pytest.mark.parametrize("seed", [50, 51])
def test_gradients_through_the_jacobian_clamp_match_central_fd(seed):
    """With x/z, y/z clamped in the EWA Jacobian (and the clamp kept by a
    margin, so the forward is smooth there), the analytic gradients of every
    parameter and of the pose equal central differences of the forward."""
    sc, P = _clamped_jacobian_scene(seed)
    wC, wD, wA = _upstream(sc, seed)
    _, g = oracle.render_backward(sc, [wC], [wD], [wA])
    clamped = np.nonzero(P["clamp_x"] + P["clamp_y"] > 0)[0]
    # the clamped Gaussians do reach the image: their parameters get gradients
    assert all(np.abs(g["means"][:, k]).max() > 1e-6 for k in clamped)
    _assert_matches_fd(g, _fd_all(sc, wC, wD, wA))


def _alpha_clamp_scene():
    """A wide, nearly opaque isotropic Gaussian A on the optical axis whose
    alpha exceeds 0.99 at exactly the four pixels around its centre (pixel
    centres at distance^2 0.5: d^2 = 0.005, sigma exp(-d^2/2) = 0.9974; the
    next ring, at distance^2 2.5, gives 0.9875), and two smaller anisotropic
    Gaussians B, C behind it."""
    c = cam(22, 22, 20.0, cx=10.5, cy=10.5)
    zA = 2.0
    sA = np.sqrt(100.0 - 0.3) * zA / 20.0                      # Sigma' = 100 I px^2
    sig_logit = np.log(0.9999 / 0.0001)
    mu = np.array([[0.0, 0.02, -0.1], [0.0, -0.05, 0.08], [zA, 3.0, 3.4]])
    ls = np.array([[np.log(sA), np.log(0.09), np.log(0.2)], [np.log(sA), np.log(0.25), np.log(0.07)],
                   [np.log(sA), np.log(0.12), np.log(0.1)]])
    q = np.array([[1.0, 0.9, 0.7], [0.0, 0.2, -0.3], [0.0, -0.3, 0.1], [0.0, 0.1, 0.5]])
    rgb = np.array([[0.7, 0.3, 0.5], [0.2, 0.8, 0.4], [0.6, 0.5, 0.9]])
    return make_scene(mu, ls, q, [sig_logit, 0.3, -0.2], dc_for_rgb(rgb), 0, [c])


def test_alpha_clamp_pixels_pass_no_gradient_through_alpha():
    """Where alpha is clamped at 0.99 it does not depend on the opacity or on
    d^2: a loss on those four pixels alone has zero gradient w.r.t. A's
    opacity logit, scales, rotation and in-plane position (A's depth still
    moves the composited depth), and central differences agree."""
    sc = _alpha_clamp_scene()
    c = sc.cameras[0]
    P = oracle.project(sc, 0)
    a_raw = P["opacity"][0] * np.exp(-0.5 * 0.5 / 100.0)
    assert a_raw > 0.99 * 1.005 and P["opacity"][0] * np.exp(-0.5 * 2.5 / 100.0) < 0.99 * 0.998
    rng = np.random.default_rng(3)
    mask = np.zeros((c.H, c.W))
    mask[10:12, 10:12] = 1.0
    wC, wD, wA = rng.uniform(-1, 1, (3, c.H, c.W)) * mask, rng.uniform(-1, 1, (c.H, c.W)) * mask, \
        rng.uniform(-1, 1, (c.H, c.W)) * mask
    out, g = oracle.render_backward(sc, [wC], [wD], [wA])
    assert (out[0]["ncontrib"][10:12, 10:12] == 3).all()
    assert g["opacity_logits"][0] == 0 and not g["log_scales"][:, 0].any() and not g["quats"][:, 0].any()
    assert not g["means"][0:2, 0].any() and g["means"][2, 0] != 0
    fd = _fd_all(sc, wC, wD, wA)
    assert abs(fd["opacity_logits"][0]) < 1e-8 and np.abs(fd["log_scales"][:, 0]).max() < 1e-8
    _assert_matches_fd(g, fd)


def test_gradients_with_alpha_clamp_match_central_fd():
    """The whole image, clamped and unclamped pixels together."""
    sc = _alpha_clamp_scene()
    out = oracle.render(sc)[0]
    assert min(out["margin"].min(), out["zmargin"].min()) > 2e-3
    wC, wD, wA = _upstream(sc, 4)
    _, g = oracle.render_backward(sc, [wC], [wD], [wA])
    _assert_matches_fd(g, _fd_all(sc, wC, wD, wA))


def test_negative_colour_is_clamped_to_zero():
    """Closed-form footprint of an isotropic Gaussian whose raw colour
    SH_0 Y_0 + 0.5 is (-0.3, 0.5, 1.2): the rendered colour is
    (0, 0.5 alpha, 1.2 alpha) -- clamped below at zero, not above at one."""
    c = cam(30, 40, 60.0)
    z, s, logit = 3.0, 0.08, 0.9
    raw = np.array([-0.3, 0.5, 1.2])
    sc = make_scene([[0.0], [0.0], [z]], np.full((3, 1), np.log(s)), [[1.0], [0.0], [0.0], [0.0]],
                    [logit], dc_for_rgb(raw)[:, None], 0, [c])
    out = oracle.render(sc)[0]
    yy, xx = np.mgrid[0:c.H, 0:c.W]
    a = _iso_alpha(1 / (1 + np.exp(-logit)), 60.0, s, z, (xx - 20.0) ** 2 + (yy - 15.0) ** 2)
    np.testing.assert_allclose(out["color"][0], 0.0, atol=0)
    np.testing.assert_allclose(out["color"][1], 0.5 * a, atol=1e-13)
    np.testing.assert_allclose(out["color"][2], 1.2 * a, atol=1e-13)


def test_clamped_colour_channel_passes_no_gradient():
    """Degree-3 colours with channel 0 of one Gaussian negative in the view
    (clamped to 0): that channel's SH coefficients get zero gradient, and
    every gradient, the view-direction terms of the other channels included,
    equals central differences."""
    rng = np.random.default_rng(60)
    while True:
        sc = _random_scene(rng, 6, 20, 24, 24.0, 3, logit_hi=2.0)
        sc.sh[0, 0] = (-0.35 - 0.5) / Y00                      # raw red of Gaussian 0 about -0.35
        out = oracle.render(sc)[0]
        P = oracle.project(sc, 0)
        colours = np.stack([P["r"], P["g"], P["b"]])
        if min(out["margin"].min(), out["zmargin"].min()) > 2e-3 and P["r"][0] == 0 and \
                np.sort(colours.reshape(-1))[1] > 0.05 and (out["ncontrib"] > 0).mean() > 0.2:
            break
    wC, wD, wA = _upstream(sc, 61)
    _, g = oracle.render_backward(sc, [wC], [wD], [wA])
    assert not g["sh"][0::3, 0].any()                           # red coefficients of Gaussian 0
    assert np.abs(g["sh"][1::3, 0]).max() > 0
    _assert_matches_fd(g, _fd_all(sc, wC, wD, wA))


def test_pose_translation_identity():
    """Moving the camera by rho equals moving every mean by W^T rho (also for
    the SH view direction), so dL/drho = W sum_g dL/dmu_g."""
    rng = np.random.default_rng(30)
    sc = _random_scene(rng, 30, 30, 40, 40.0, 3, logit_hi=3.0)
    wC, wD, wA = _upstream(sc, 31)
    _, g = oracle.render_backward(sc, [wC], [wD], [wA])
    W = sc.cameras[0].T_cw[:, :3]
    np.testing.assert_allclose(g["pose"][0, :3], W @ g["means"].sum(1), rtol=1e-10, atol=1e-12)


def test_pixel_subset_matches_full_image():
    """Gradients of a loss on a pixel subset equal the full-image gradients of
    the same loss with zero weight elsewhere."""
    rng = np.random.default_rng(40)
    sc = _random_scene(rng, 30, 20, 30, 30.0, 3)
    c = sc.cameras[0]
    pix = np.sort(rng.choice(c.H * c.W, 70, replace=False))
    gC = rng.uniform(-1, 1, (3, 70)); gD = rng.uniform(-1, 1, 70); gA = rng.uniform(-1, 1, 70)
    fC = np.zeros((3, c.H * c.W)); fD = np.zeros(c.H * c.W); fA = np.zeros(c.H * c.W)
    fC[:, pix] = gC; fD[pix] = gD; fA[pix] = gA
    o1, g1 = oracle.render_backward(sc, [gC], [gD], [gA], pixels=[pix])
    o2, g2 = oracle.render_backward(sc, [fC.reshape(3, c.H, c.W)], [fD.reshape(c.H, c.W)],
                                    [fA.reshape(c.H, c.W)])
    for k in ("means", "log_scales", "quats", "opacity_logits", "sh", "pose"):
        np.testing.assert_allclose(g1[k], g2[k], rtol=1e-12, atol=1e-14)
    np.testing.assert_array_equal(o1[0]["color"], o2[0]["color"].reshape(3, -1)[:, pix])


# ---------------------------------------------------------------- median depth

def test_median_depth_worked_cases():
    """Two Gaussians on the axis: the median is the front one's depth where it
    alone takes the accumulated opacity past 0.5, else the one behind it."""
    c = cam(9, 9, 50.0)
    z1, z2 = 2.0, 3.0
    sig = lambda l: 1 / (1 + np.exp(-l))
    for l1, expect_front in ((3.0, True), (-1.0, False)):
        sc = make_scene([[0.0, 0.0], [0.0, 0.0], [z2, z1]], np.log([[0.08, 0.04]] * 3),
                        [[1.0, 1.0], [0, 0], [0, 0], [0, 0]], [1.2, l1],
                        np.stack([dc_for_rgb([0.5] * 3), dc_for_rgb([0.5] * 3)], 1), 0, [c])
        out = oracle.render(sc)[0]
        for (x, y) in [(4, 4), (5, 5)]:
            r2 = (x - 4.5) ** 2 + (y - 4.5) ** 2
            a1 = float(_iso_alpha(sig(l1), 50.0, 0.04, z1, r2))
            a2 = float(_iso_alpha(sig(1.2), 50.0, 0.08, z2, r2))
            assert (1 - a1 < 0.5) == expect_front
            want = z1 if (1 - a1 <= 0.5 or a2 == 0) else z2
            assert out["median_depth"][y, x] == want
    # no contributor: zero
    sc = make_scene([[0.0], [0.0], [-3.0]], np.log([[0.05]] * 3), [[1.0], [0], [0], [0]], [1.0],
                    dc_for_rgb([0.5] * 3)[:, None], 0, [c])
    assert not oracle.render(sc)[0]["median_depth"].any()


def test_median_depth_brute_force_from_projection():
    """Per pixel, from the oracle's projected quantities alone: evaluate every
    Gaussian's alpha with the skip/clamp/stop rules in (z, index) order and
    take the z of the last contributor entered with transmittance above 0.5."""
    rng = np.random.default_rng(21)
    sc = _random_scene(rng, 12, 16, 20, 20.0, 0)
    out = oracle.render(sc)[0]
    P = oracle.project(sc, 0)
    order = sorted(range(12), key=lambda g: (P["z"][g], g))
    c = sc.cameras[0]
    checked = 0
    for y in range(c.H):
        for x in range(c.W):
            if out["median_margin"][y, x] < 1e-6:
                continue
            T, med = 1.0, 0.0
            for g in order:
                if not P["valid"][g]:
                    continue
                dx, dy = x - P["u"][g], y - P["v"][g]
                d2 = P["conic0"][g] * dx * dx + 2 * P["conic1"][g] * dx * dy + P["conic2"][g] * dy * dy
                if d2 > 9:
                    continue
                a = P["opacity"][g] * np.exp(-0.5 * d2)
                if a < 1 / 255:
                    continue
                a = min(a, 0.99)
                if T * (1 - a) < 1e-4:
                    break
                if T > 0.5:
                    med = P["z"][g]
                T *= 1 - a
            assert out["median_depth"][y, x] == pytest.approx(med, abs=1e-12)
            checked += 1
    assert checked > 0.9 * c.H * c.W


def test_median_depth_gradient_matches_central_fd():
    rng = np.random.default_rng(5)
    while True:
        sc = _fd_scene(int(rng.integers(100, 10_000)), deg=0)
        o = oracle.render(sc)[0]
        if o["median_margin"].min() > 2e-3 and (o["median_depth"] > 0).mean() > 0.2:
            break
    c = sc.cameras[0]
    wM = rng.uniform(-1, 1, (c.H, c.W))
    zero = np.zeros((c.H, c.W))
    _, g = oracle.render_backward(sc, [np.zeros((3, c.H, c.W))], [zero], [zero], gM=[wM])
    h = 1e-6
    fd = np.zeros_like(sc.means)
    for i in range(sc.means.size):
        flat = sc.means.reshape(-1)
        keep = flat[i]
        flat[i] = keep + h
        lp = (wM * oracle.render(sc)[0]["median_depth"]).sum()
        flat[i] = keep - h
        lm = (wM * oracle.render(sc)[0]["median_depth"]).sum()
        flat[i] = keep
        fd.reshape(-1)[i] = (lp - lm) / (2 * h)
    err = np.linalg.norm(g["means"] - fd) / max(np.linalg.norm(fd), 1e-30)
    assert err < 1e-6
    # nothing else moves the median: the other parameters get no gradient
    for k in ("log_scales", "quats", "opacity_logits", "sh"):
        assert not g[k].any(), k


# ---------------------------------------------------------------- densification statistics

def test_densify_stats_single_gaussian_closed_form():
    """One isotropic Gaussian on the axis: visible in the view, radius
    3 sqrt((f s/z)^2 + 0.3), and |dL/du| of L = sum_p w_p C_r(p) from the
    closed-form footprint: dC_r/du = c alpha (x - u)/var."""
    c = cam(40, 48, 80.0)
    z, s, logit = 3.0, 0.06, 0.8
    rgb = np.array([0.7, 0.2, 0.4])
    sc = make_scene([[0.0], [0.0], [z]], np.full((3, 1), np.log(s)), [[1.0], [0.0], [0.0], [0.0]],
                    [logit], dc_for_rgb(rgb)[:, None], 0, [c])
    rng = np.random.default_rng(2)
    wr = rng.uniform(-1, 1, (c.H, c.W))
    gC = np.stack([wr, np.zeros_like(wr), np.zeros_like(wr)])
    zero = np.zeros((c.H, c.W))
    _, g = oracle.render_backward(sc, [gC], [zero], [zero], want_screen=True)
    st = oracle.densify_stats(sc, g["screen"])
    var = (80.0 * s / z) ** 2 + 0.3
    yy, xx = np.mgrid[0:c.H, 0:c.W]
    r2 = (xx - 24.0) ** 2 + (yy - 20.0) ** 2
    a = _iso_alpha(1 / (1 + np.exp(-logit)), 80.0, s, z, r2)
    dudx = (wr * rgb[0] * a * (xx - 24.0) / var).sum()
    dvdy = (wr * rgb[0] * a * (yy - 20.0) / var).sum()
    assert st["count"][0] == 1
    assert st["radius"][0] == pytest.approx(3 * np.sqrt(var), rel=1e-12)
    assert st["grad"][0] == pytest.approx(np.hypot(dudx, dvdy), rel=1e-10)


def test_densify_stats_visibility_and_sums_over_views():
    """Visible views are counted once each, the gradient norms add up, the
    radius is the largest; a Gaussian behind every camera has no statistics."""
    rng = np.random.default_rng(8)
    sc = _random_scene(rng, 10, 18, 22, 22.0, 0)
    c0 = sc.cameras[0]
    far = scenes.Camera(c0.H, c0.W, c0.fx, c0.fy, c0.cx, c0.cy,
                        np.hstack([np.eye(3), [[0.0], [0.0], [0.7]]]))
    sc = sc.with_cameras([c0, far])
    gC, gD, gA = (rng.uniform(-1, 1, (3, c0.H, c0.W)), rng.uniform(-1, 1, (c0.H, c0.W)),
                  rng.uniform(-1, 1, (c0.H, c0.W)))
    _, g = oracle.render_backward(sc, [gC, gC], [gD, gD], [gA, gA], want_screen=True)
    st = oracle.densify_stats(sc, g["screen"])
    per = [oracle.densify_stats(sc.with_cameras([cc]), g["screen"][v:v + 1]) for v, cc in enumerate(sc.cameras)]
    np.testing.assert_allclose(st["grad"], per[0]["grad"] + per[1]["grad"], rtol=1e-12)
    np.testing.assert_array_equal(st["count"], per[0]["count"] + per[1]["count"])
    np.testing.assert_allclose(st["radius"], np.maximum(per[0]["radius"], per[1]["radius"]), rtol=1e-12)
    # a Gaussian with a screen gradient is visible in that view
    for v in range(2):
        moved = np.hypot(g["screen"][v][0], g["screen"][v][1]) > 0
        assert (per[v]["count"][moved] == 1).all()
    # behind the camera: nothing
    sc2 = make_scene([[0.0], [0.0], [-2.0]], np.full((3, 1), -3.0), [[1.0], [0], [0], [0]], [1.0],
                     dc_for_rgb([0.5] * 3)[:, None], 0, [c0])
    st2 = oracle.densify_stats(sc2, np.zeros((1, 10, 1)))
    assert st2["count"][0] == 0 and st2["grad"][0] == 0 and st2["radius"][0] == 0


def test_densify_box_visibility_brute_force():
    """The box minimum of the quadratic equals a dense grid search (to the
    grid's resolution), inside and outside the box."""
    rng = np.random.default_rng(4)
    for _ in range(40):
        A = rng.normal(size=(2, 2))
        S = A @ A.T + 0.1 * np.eye(2)
        a, b, d = np.linalg.inv(S)[0, 0], np.linalg.inv(S)[0, 1], np.linalg.inv(S)[1, 1]
        u, v = rng.uniform(-6, 16, 2)
        q = oracle._quad_min_over_box(a, b, d, u, v, 0.0, 9.0, 0.0, 7.0)
        xs, ys = np.meshgrid(np.linspace(0, 9, 901), np.linspace(0, 7, 701))
        dx, dy = xs - u, ys - v
        grid = (a * dx * dx + 2 * b * dx * dy + d * dy * dy).min()
        assert q <= grid + 1e-12
        assert q == pytest.approx(grid, rel=2e-3, abs=2e-4)
