"""GPU parity of the CUDA rasteriser against the FP64 oracle (through the C ABI).

Sizes: the five workloads at reduced sizes that the oracle renders in
seconds (several tiles, ragged right/bottom edges), and at full size on
sampled pixels (forward) and with upstream gradients that are zero except on
sampled pixels (backward: the oracle then needs only those pixels)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2411_17660_b300 import binding as B
from paper_2411_17660_b300 import render as R
from paper_2411_17660_b300 import scenes
from tests import gsr_testutil as U

pytestmark = pytest.mark.gpu

REDUCED = {
    "small": lambda: scenes.config_small(),
    "room": lambda: scenes.config_room(N=4000, H=140, W=250, f=125.0),
    "window": lambda: scenes.config_window(N=5000, V=4, H=75, W=100, f=78.0),
    "uneven": lambda: scenes.config_uneven(N=8000, V=5, res_scale=0.15),
    "outdoor": lambda: scenes.config_outdoor(N=10000, V=3, H=108, W=190, f=140.0),
}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("name", list(REDUCED))
def test_forward_parity_reduced(name):
    sc = REDUCED[name]()
    got, _ = U.gpu_forward(sc)
    ref = oracle.render(sc)
    flips = total = near = 0
    for v, (r, g) in enumerate(zip(ref, got)):
        f, n, e = U.compare_images(r, g, f"{name} view {v}")
        flips, total, near = flips + f, total + n, near + e["near_threshold"]
    assert flips <= max(2, U.FLIP_SHARE * total), f"{flips} threshold-flip pixels of {total}"
    # the per-pixel tolerance holds on all but a small share of the pixels
    assert near <= 0.01 * total, f"{near} of {total} pixels near a threshold"


@pytest.mark.parametrize("name", list(REDUCED))
def test_backward_parity_reduced(name):
    sc = REDUCED[name]()
    _, state = U.gpu_forward(sc)
    gC, gD, gA = U.upstream(sc)
    got = U.gpu_backward(sc, state, gC, gD, gA)
    _, ref = oracle.render_backward(sc, gC, gD, gA)
    U.compare_grads(ref, got, label=name)


def _opaque_stack(seed=31, N=2500, H=60, W=80, f=70.0):
    """A dense stack of nearly opaque Gaussians in front of one view, so that
    most pixels meet the transmittance stop part-way down their lists."""
    import dataclasses
    rng = np.random.default_rng(seed)
    base = scenes.config_small(seed=seed, N=N, H=H, W=W, f=f)
    z = rng.uniform(2.0, 5.0, N)
    xy = rng.uniform(-0.9, 0.9, (2, N)) * z * np.array([[W / (2 * f)], [H / (2 * f)]])
    return dataclasses.replace(
        base, means=np.ascontiguousarray(np.stack([xy[0], xy[1], z]).astype(np.float32)),
        log_scales=np.ascontiguousarray(rng.normal(-1.9, 0.3, (3, N)).astype(np.float32)),
        opacity_logits=np.ascontiguousarray(rng.normal(4.0, 0.5, N).astype(np.float32)))


def test_transmittance_stop_forward_and_backward():
    """Pixels that stop part-way down their lists: the forward keeps the stop
    position, and the backward's contributors (the entries before it that
    reach the pixel) give the oracle's gradients."""
    sc = _opaque_stack()
    got, state = U.gpu_forward(sc)
    ref = oracle.render(sc)
    stopped = ref[0]["T"] < 2e-4
    assert stopped.mean() > 0.3, "most pixels should meet the stop"
    n_ref = int(ref[0]["ncontrib"].sum())
    U.compare_images(ref[0], got[0], "opaque stack")
    info = state[0].info(state[4])
    flips = (ref[0]["margin"] < U.MARGIN) | (ref[0]["zmargin"] < U.ZMARGIN)
    # composited pairs counted by the forward = the oracle's contributors (up to flips)
    assert abs(info.pairs_contributing - n_ref) <= int(flips.sum()) * 4
    gC, gD, gA = U.upstream(sc)
    g = U.gpu_backward(sc, state, gC, gD, gA)
    _, gref = oracle.render_backward(sc, gC, gD, gA)
    U.compare_grads(gref, g, label="opaque stack")


def _axis_band(seed=37, N=1500, H=60, W=96, f=70.0):
    """Unrotated Gaussians whose means lie on the camera's y = 0 plane: their
    projected covariances have an exactly zero off-diagonal (m01 = 0), so a
    row that has met the stop evaluates 0 times its far row offset.  The left
    half of the band is translucent (opacity about 0.92: its tiles' chunks skip
    the 0.99 clamp), the right half opaque (above 0.99: clamped chunks); both
    are dense enough that most band pixels meet the transmittance stop."""
    import dataclasses
    rng = np.random.default_rng(seed)
    base = scenes.config_small(seed=seed, N=N, H=H, W=W, f=f)
    while True:
        z = rng.uniform(2.0, 5.0, N)
        if scenes.distinct_f32(z):
            break
    u = rng.uniform(-0.95, 0.95, N)
    x = u * z * W / (2 * f)
    logit = np.where(u < 0.0, rng.normal(2.5, 0.2, N), rng.normal(5.5, 0.3, N))
    quats = np.zeros((4, N), np.float32)
    quats[0] = rng.uniform(0.5, 2.0, N)   # unnormalised identity rotations
    return dataclasses.replace(
        base, means=np.ascontiguousarray(np.stack([x, np.zeros(N), z]).astype(np.float32)),
        log_scales=np.ascontiguousarray(rng.normal(-2.0, 0.25, (3, N)).astype(np.float32)),
        quats=quats, opacity_logits=np.ascontiguousarray(logit.astype(np.float32)))


def test_stop_with_zero_off_diagonal_and_both_clamp_paths():
    """Stopped rows with m01 = 0, and chunks with and without a Gaussian that
    reaches the alpha clamp: finite images equal to the oracle's, forward and
    backward, and the oracle sees both opacity ranges composited."""
    sc = _axis_band()
    got, state = U.gpu_forward(sc)
    for key in ("color", "depth", "alpha"):
        assert np.isfinite(got[0][key]).all(), key
    ref = oracle.render(sc)
    assert (ref[0]["T"] < 2e-4).mean() > 0.15, "band pixels should meet the stop"
    U.compare_images(ref[0], got[0], "axis band")
    gC, gD, gA = U.upstream(sc)
    g = U.gpu_backward(sc, state, gC, gD, gA)
    for k, v in g.items():
        assert np.isfinite(v).all(), k
    _, gref = oracle.render_backward(sc, gC, gD, gA)
    U.compare_grads(gref, g, label="axis band")


def _edge_stress(seed=41, N=3000, H=48, W=64, f=60.0):
    """Gaussians around the image borders (centres from 0.6 image widths
    outside to 0.6 inside past the far edge), beyond the Jacobian clamp, and
    at the near plane, anisotropic with opacities across the alpha cutoff,
    seen by three cameras 2.6 km from the world origin (large coordinates
    whose camera transform cancels).  The forward's conservative cull must
    keep every pair whose cutoff ellipse reaches a pixel centre."""
    import dataclasses
    from scipy.spatial.transform import Rotation
    rng = np.random.default_rng(seed)
    base = scenes.config_small(seed=seed, N=N, H=H, W=W, f=f)
    near = rng.uniform(size=N) < 0.2
    z = np.where(near, rng.uniform(0.19, 0.26, N), rng.uniform(0.3, 8.0, N))
    u = rng.uniform(-0.6 * W, 1.6 * W, N)
    v = rng.uniform(-0.6 * H, 1.6 * H, N)
    O = np.array([2000.0, -700.0, 1500.0])
    means = np.stack([(u - W / 2) * z / f, (v - H / 2) * z / f, z]) + O[:, None]
    rots = [np.eye(3), Rotation.from_rotvec([0.0, 0.3, 0.0]).as_matrix(),
            Rotation.from_rotvec([-0.25, 0.0, 0.2]).as_matrix()]
    centres = [O, O + np.array([0.5, 0.2, -0.3]), O + np.array([-0.3, 0.1, 0.2])]
    cams = [scenes.Camera(H, W, f, f, W / 2, H / 2, scenes.pose_from_c2w(Rm, C)) for Rm, C in zip(rots, centres)]
    sc = dataclasses.replace(
        base, means=np.ascontiguousarray(means.astype(np.float32)),
        log_scales=np.ascontiguousarray(np.minimum(rng.normal(-2.5, 1.0, (3, N)), 0.5).astype(np.float32)),
        quats=np.ascontiguousarray(rng.normal(size=(4, N)).astype(np.float32)),
        opacity_logits=np.ascontiguousarray(rng.normal(0.0, 3.0, N).astype(np.float32)))
    return sc.with_cameras(cams)


def test_conservative_cull_keeps_every_reaching_pair():
    """The preprocess culls (view, Gaussian) pairs with FP32 bounds before
    the exact projection: on pairs placed at the borders, past the Jacobian
    clamp and at the near plane, the images equal the oracle's and so does
    every Gaussian's count of views whose cutoff ellipse reaches a pixel
    centre (a culled pair gets radius 0)."""
    sc = _edge_stress()
    got, state = U.gpu_forward(sc)
    ref = oracle.render(sc)
    for v in range(sc.V):
        U.compare_images(ref[v], got[v], f"edge stress view {v}")
    # the scene reaches the cases: visible pairs centred outside the image,
    # clamped ones, near-plane ones
    outside = clamped = near = 0
    for c in sc.cameras:
        P = oracle.project(sc, camera=c)
        for g in np.nonzero(P["valid"])[0]:
            d2max = min(9.0, 2.0 * np.log(255.0 * P["opacity"][g]))
            if not d2max >= 0:
                continue
            q = oracle._quad_min_over_box(P["conic0"][g], P["conic1"][g], P["conic2"][g], P["u"][g], P["v"][g],
                                          0.0, c.W - 1.0, 0.0, c.H - 1.0)
            if q > d2max:
                continue
            outside += not (0 <= P["u"][g] <= c.W - 1 and 0 <= P["v"][g] <= c.H - 1)
            clamped += bool(P["clamp_x"][g] or P["clamp_y"][g])
            near += P["z"][g] < 0.26
    assert outside > 300 and clamped > 100 and near > 20, (outside, clamped, near)
    rast, params, cams, vm, ws, color, depth, alpha = state
    gC, gD, gA = U.upstream(sc)
    flat = lambda arrs: torch.from_numpy(np.concatenate([np.asarray(a, np.float32).reshape(-1) for a in arrs])).cuda()
    dens = {k: torch.full((sc.N,), np.nan, device="cuda") for k in ("grad", "count", "radius")}
    grads = {k: torch.empty_like(x) for k, x in params.items()}
    rast.backward_raw(params, sc.sh_degree, cams, vm, ws, flat(gC), flat(gD), flat(gA), grads, None, densify=dens)
    torch.cuda.synchronize()
    count = dens["count"].cpu().numpy()
    _, rg = oracle.render_backward(sc, gC, gD, gA, want_screen=True)
    ref_d = oracle.densify_stats(sc, rg["screen"])
    sure = ref_d["margin"] > 1e-3
    assert sure.mean() > 0.99
    np.testing.assert_array_equal(count[sure], ref_d["count"][sure])


def test_gradient_rows_clean_record():
    """The forward clears the screen-gradient rows only when the workspace
    header does not record this layout's rows as clean.  A workspace of
    garbage, a surfel forward and backward (whose rows stay filled) in
    between, a smaller Gaussian set on the same workspace, and back-to-back
    iterations all give the gradients of a fresh workspace."""
    sc = REDUCED["window"]()
    gC, gD, gA = U.upstream(sc)
    _, ref_state = U.gpu_forward(sc)
    ref = U.gpu_backward(sc, ref_state, gC, gD, gA)
    rast, params, cams, vm, ws = ref_state[:5]

    def step(scene, prm, ws):
        color, depth, alpha, ws2 = rast.render_forward(prm, scene.sh_degree, cams, vm, ws=ws, grow=False)
        assert ws2 is ws and rast.info(ws).status == B.OK
        return U.gpu_backward(scene, (rast, prm, cams, vm, ws, color, depth, alpha), gC, gD, gA)

    def same(a, b, label):
        for k in a:
            assert U.rel_l2(b[k], a[k]) < 1e-5, (label, k, U.rel_l2(b[k], a[k]))

    ws.fill_(255)   # every float NaN, no record
    same(ref, step(sc, params, ws), "garbage workspace")
    same(ref, step(sc, params, ws), "second iteration")
    P = R.pixel_offsets(cams)[-1]
    bufs = [torch.empty(n * P, device="cuda") for n in (3, 1, 1, 3, 1)]
    rast.surfels_forward_raw(params, sc.sh_degree, cams, vm, ws, *bufs)
    ups = [torch.rand(n * P, device="cuda") - 0.5 for n in (3, 1, 1, 3, 1)]
    sg = {k: torch.empty_like(x) for k, x in params.items()}
    rast.surfels_backward_raw(params, sc.sh_degree, cams, vm, ws, *ups, sg, None)
    same(ref, step(sc, params, ws), "after surfels")
    sub = sc.subset(np.arange(0, sc.N, 2))
    _, sub_state = U.gpu_forward(sub)
    sub_ref = U.gpu_backward(sub, sub_state, gC, gD, gA)
    sub_params = U.to_device(sub)[0]
    same(sub_ref, step(sub, sub_params, ws), "smaller set, same workspace")
    same(ref, step(sc, params, ws), "full set again")


@pytest.mark.parametrize("tile,binning,rows", [(8, "tile", 8), (16, "tile", 16), (16, "tile", 8), (32, "tile", 16),
                                               (32, "tile", 8), (16, "radix", 16)])
def test_decisions_backward_equals_forward(tile, binning, rows):
    """The checked build counts the backward's contributor pairs: they are
    exactly the forward's composited pairs (both kernels form every s with
    the same FP32 operations), at every tile size, also where pixels stop."""
    if not B.LIB_PATH.endswith("libgsr_checked.so"):
        pytest.skip("the backward's pair count is kept by the checked build (tests/test_checked_gpu.py)")
    for sc in (REDUCED["window"](), REDUCED["uneven"](), REDUCED["outdoor"](), _opaque_stack(), _axis_band()):
        _, state = U.gpu_forward(sc, rast=R.GaussianRasterizer(tile, binning=binning, fwd_rows=rows))
        gC, gD, gA = U.upstream(sc)
        U.gpu_backward(sc, state, gC, gD, gA)
        info = state[0].info(state[4])
        assert info.status == B.OK
        assert info.pairs_backward == info.pairs_contributing > 0, (sc.name, info.pairs_backward,
                                                                     info.pairs_contributing)


def test_tile_size_invariance():
    """Tile size and the forward's warp-block height change which entries a
    warp stages, never a pixel's arithmetic: bit-identical images."""
    sc = REDUCED["room"]()
    outs = [U.gpu_forward(sc, tile=t)[0][0] for t in (8, 16, 32)]
    outs += [U.gpu_forward(sc, rast=R.GaussianRasterizer(t, fwd_rows=8))[0][0] for t in (16, 32)]
    for o in outs[1:]:
        for k in ("color", "depth", "alpha"):
            np.testing.assert_array_equal(o[k], outs[0][k])


def test_batched_equals_per_view():
    sc = REDUCED["window"]()
    batched, state = U.gpu_forward(sc)
    gC, gD, gA = U.upstream(sc)
    gb = U.gpu_backward(sc, state, gC, gD, gA)
    acc = None
    for v in range(sc.V):
        one = sc.with_cameras([sc.cameras[v]], [sc.target_color[v]], [sc.target_depth[v]])
        single, st1 = U.gpu_forward(one)
        for k in ("color", "depth", "alpha"):
            np.testing.assert_array_equal(single[0][k], batched[v][k])
        g1 = U.gpu_backward(one, st1, [gC[v]], [gD[v]], [gA[v]])
        np.testing.assert_allclose(g1["pose"][0], gb["pose"][v], rtol=1e-4, atol=1e-6)
        if acc is None:
            acc = {k: g1[k].copy() for k in g1 if k != "pose"}
        else:
            for k in acc:
                acc[k] += g1[k]
    for k in acc:
        assert U.rel_l2(gb[k], acc[k]) < 1e-5, k


def test_permutation_invariance():
    sc = REDUCED["room"]()
    perm = np.random.default_rng(0).permutation(sc.N)
    a = U.gpu_forward(sc)[0][0]
    b = U.gpu_forward(sc.subset(perm))[0][0]
    for k in ("color", "depth", "alpha"):
        np.testing.assert_array_equal(a[k], b[k])


def test_capacity_overflow_is_reported_then_grown():
    sc = REDUCED["uneven"]()
    rast = R.GaussianRasterizer(16)
    params, cams, vm = U.to_device(sc)
    _, _, _, ws = rast.render_forward(params, sc.sh_degree, cams, vm)
    assert rast.info(ws).keys > 2 * 3072, "needs more keys than the smallest capacity"
    rast = R.GaussianRasterizer(16)
    small = rast.alloc_workspace(sc.N, cams, key_capacity=3072)
    P = sum(c.H * c.W for c in cams)
    color = torch.empty(3 * P, device="cuda")
    rast.forward_raw(params, sc.sh_degree, cams, vm, small, color, None, None)
    info = rast.info(small)
    assert info.status == B.ECAPACITY and info.keys > info.key_capacity
    assert rast.ctx.get_status(small.data_ptr(), small.numel(), torch.cuda.current_stream().cuda_stream) == \
        B.ECAPACITY
    c2, _, _, ws = rast.render_forward(params, sc.sh_degree, cams, vm)
    assert rast.ctx.get_status(ws.data_ptr(), ws.numel(), torch.cuda.current_stream().cuda_stream) == B.OK
    assert rast.info(ws).status == B.OK
    ref = U.gpu_forward(sc)[0]
    for v, c in enumerate(R.split_views(c2, cams, 3)):
        np.testing.assert_array_equal(c.cpu().numpy(), ref[v]["color"])


def test_bounded_lookback_gives_up_with_status():
    """Test hook (radix binning): the first sort tile never publishes its digit counts, so the
    next tile's bounded wait must run out and report GSR_ETIMEOUT; the
    context and the device stay usable."""
    sc = REDUCED["uneven"]()
    params, cams, vm = U.to_device(sc)
    ok = R.GaussianRasterizer(16, binning="radix")
    _, _, _, ws = ok.render_forward(params, sc.sh_degree, cams, vm)
    assert ok.info(ws).keys > 2 * 3072, "needs at least two sort tiles"
    stall = R.GaussianRasterizer(16, spin_limit=2000, flags=B.TEST_STALL_SORT, binning="radix")
    P = sum(c.H * c.W for c in cams)
    color = torch.empty(3 * P, device="cuda")
    stall.forward_raw(params, sc.sh_degree, cams, vm, ws, color, None, None)
    assert stall.info(ws).status == B.ETIMEOUT
    c2, _, _, ws2 = ok.render_forward(params, sc.sh_degree, cams, vm)
    assert ok.info(ws2).status == B.OK


def test_nan_gaussian_is_culled():
    sc = REDUCED["small"]()
    bad = sc.subset(np.arange(sc.N))
    bad.means[:, 7] = np.nan
    bad.log_scales[:, 9] = np.inf
    got = U.gpu_forward(bad)[0][0]
    ref = oracle.render(sc.subset(np.setdiff1d(np.arange(sc.N), [7, 9])))[0]
    U.compare_images(ref, got, "nan")


def test_autograd_function_matches_raw_backward():
    sc = REDUCED["window"]()
    params, cams, vm = U.to_device(sc)
    rast = R.GaussianRasterizer(16)
    leaves = {k: v.clone().requires_grad_(True) for k, v in params.items()}
    tangent = torch.zeros(len(cams), 6, device="cuda", requires_grad=True)
    color, depth, alpha = rast.render(leaves["means"], leaves["log_scales"], leaves["quats"],
                                      leaves["opacity_logits"], leaves["sh"], sc.sh_degree, cams, vm, tangent)
    gC, gD, gA = U.upstream(sc)
    flat = lambda arrs: torch.from_numpy(np.concatenate([np.asarray(a, np.float32).reshape(-1) for a in arrs])).cuda()
    loss = (color * flat(gC)).sum() + (depth * flat(gD)).sum() + (alpha * flat(gA)).sum()
    loss.backward()
    _, state = U.gpu_forward(sc)
    raw = U.gpu_backward(sc, state, gC, gD, gA)
    for k in R.PARAM_NAMES:
        assert U.rel_l2(leaves[k].grad.cpu().numpy().astype(np.float64), raw[k]) < 1e-5, k
    assert U.rel_l2(tangent.grad.cpu().numpy().astype(np.float64), raw["pose"]) < 1e-5


def test_l1_loss_front_end():
    sc = REDUCED["window"]()
    _, state = U.gpu_forward(sc)
    rast, params, cams, vm, ws, color, depth, alpha = state
    tc = torch.from_numpy(np.concatenate([t.reshape(-1) for t in sc.target_color])).cuda()
    td = torch.from_numpy(np.concatenate([t.reshape(-1) for t in sc.target_depth])).cuda()
    dC, dD = torch.empty_like(color), torch.empty_like(depth)
    loss = torch.empty(1, device="cuda")
    R.l1_loss(rast, cams, vm, color, depth, tc, td, 1.0, 0.1, dC, dD, loss)
    torch.cuda.synchronize()
    off = R.pixel_offsets(cams)
    exp_loss, eC, eD = 0.0, [], []
    c64, d64 = color.double().cpu(), depth.double().cpu()
    tc64, td64 = tc.double().cpu(), td.double().cpu()
    for v in range(len(cams)):
        P = off[v + 1] - off[v]
        dc = c64[3 * off[v]:3 * off[v + 1]] - tc64[3 * off[v]:3 * off[v + 1]]
        dd = d64[off[v]:off[v + 1]] - td64[off[v]:off[v + 1]]
        exp_loss += dc.abs().sum().item() / (3 * P) + 0.1 * dd.abs().sum().item() / P
        eC.append(torch.sign(dc) / (3 * P))
        eD.append(0.1 * torch.sign(dd) / P)
    assert loss.item() == pytest.approx(exp_loss, rel=1e-5)
    np.testing.assert_allclose(dC.cpu().numpy(), torch.cat(eC).numpy(), rtol=1e-6, atol=1e-12)
    np.testing.assert_allclose(dD.cpu().numpy(), torch.cat(eD).numpy(), rtol=1e-6, atol=1e-12)


# ------------------------------------------------------------------ full size

FULL = {
    "room": lambda: scenes.config_room(),
    "window": lambda: scenes.config_window(),
    "uneven": lambda: scenes.config_uneven(),
    "outdoor": lambda: scenes.config_outdoor(),
}


@pytest.mark.parametrize("name", list(FULL))
def test_full_size_sampled_pixels(name):
    sc = FULL[name]()
    per_view = {"room": 400, "window": 150, "uneven": 60, "outdoor": 24}[name]
    pix, gCs, gDs, gAs = scenes.sparse_pixel_grads(sc, per_view, seed=11)
    got, state = U.gpu_forward(sc)
    ref = oracle.render(sc, pixels=pix, brute=True)
    flips = total = near = 0
    for v, (r, g) in enumerate(zip(ref, got)):
        sel = {k: (g[k].reshape(3, -1)[:, pix[v]] if k == "color" else g[k].reshape(-1)[pix[v]])
               for k in ("color", "depth", "alpha")}
        f, n, e = U.compare_images(r, sel, f"{name} view {v}")
        flips, total, near = flips + f, total + n, near + e["near_threshold"]
    assert flips <= max(2, U.FLIP_SHARE * total * 10), f"{flips} threshold-flip pixels of {total}"
    # deep lists at full size: more close depth pairs per pixel, still a small share
    assert near <= 0.05 * total, f"{near} of {total} pixels near a threshold"
    # sparse upstream gradients: dense on the GPU, listed pixels for the oracle
    gC, gD, gA = [], [], []
    for v, c in enumerate(sc.cameras):
        a = np.zeros((3, c.H * c.W), np.float32); a[:, pix[v]] = gCs[v]; gC.append(a.reshape(3, c.H, c.W))
        d = np.zeros(c.H * c.W, np.float32); d[pix[v]] = gDs[v] * 0.1; gD.append(d.reshape(c.H, c.W))
        e = np.zeros(c.H * c.W, np.float32); e[pix[v]] = gAs[v]; gA.append(e.reshape(c.H, c.W))
    gpu = U.gpu_backward(sc, state, gC, gD, gA)
    _, orc = oracle.render_backward(sc, gCs, [g * 0.1 for g in gDs], gAs, pixels=pix, brute=True)
    U.compare_grads(orc, gpu, label=name)


GRAPH_SCENES = {
    "window": lambda: REDUCED["window"](),
    # an uneven batch: 16 keyframes of resolutions drawn from {320x240, 640x480, 1200x680} (scaled by 0.3)
    "uneven16": lambda: scenes.config_uneven(N=30000, V=16, res_scale=0.3),
}


@pytest.mark.parametrize("name,binning,fused", [("window", "tile", False), ("window", "tile", True),
                                                ("uneven16", "tile", True), ("uneven16", "radix", True)])
def test_cuda_graph_replay_matches_eager(name, binning, fused):
    """Forward + loss + backward captured once in a CUDA graph, replayed on
    changed inputs (same buffers), equals the eager calls on those inputs;
    fused: the L1 loss taken in the forward blend (gsr_render_l1), as the
    benchmark runs it.  uneven16: a 16-keyframe batch of mixed resolutions,
    with both binning strategies (the radix one is the autotuner's choice for
    the full-size uneven batch)."""
    sc = GRAPH_SCENES[name]()
    assert name != "uneven16" or (sc.V == 16 and len({(c.H, c.W) for c in sc.cameras}) == 3)
    rast = R.GaussianRasterizer(16, binning=binning)
    params, cams, vm = U.to_device(sc)
    color, depth, alpha, ws = rast.render_forward(params, sc.sh_degree, cams, vm)
    ws = rast.alloc_workspace(sc.N, cams, int(rast.info(ws).keys * 2) + 8192)
    tc = torch.from_numpy(np.concatenate([t.reshape(-1) for t in sc.target_color])).cuda()
    td = torch.from_numpy(np.concatenate([t.reshape(-1) for t in sc.target_depth])).cuda()
    dC, dD = torch.empty_like(color), torch.empty_like(depth)
    loss = torch.empty(1, device="cuda")
    grads = {k: torch.empty_like(v) for k, v in params.items()}
    d_pose = torch.empty(len(cams), 6, device="cuda")

    def step():
        if fused:
            rast.forward_l1_raw(params, sc.sh_degree, cams, vm, ws, color, depth, alpha, tc, td, 1.0, 0.1, dC, dD,
                                loss)
        else:
            rast.forward_raw(params, sc.sh_degree, cams, vm, ws, color, depth, alpha)
            R.l1_loss(rast, cams, vm, color, depth, tc, td, 1.0, 0.1, dC, dD, loss)
        rast.backward_raw(params, sc.sh_degree, cams, vm, ws, dC, dD, None, grads, d_pose)

    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        step()
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        step()
    # new inputs in the same buffers: move the Gaussians and the cameras a bit
    with torch.no_grad():
        params["means"].add_(0.01)
        vm[:, :, 3].add_(0.02)
    graph.replay()
    torch.cuda.synchronize()
    got = {k: v.clone() for k, v in grads.items()}
    got_img, got_pose, got_loss = color.clone(), d_pose.clone(), loss.clone()
    assert rast.info(ws).status == B.OK
    step()
    torch.cuda.synchronize()
    assert torch.equal(color, got_img)
    assert torch.allclose(loss, got_loss, rtol=1e-5)
    for k in R.PARAM_NAMES:
        assert U.rel_l2(got[k].cpu().numpy().astype(np.float64), grads[k].cpu().numpy().astype(np.float64)) < 1e-5
    assert U.rel_l2(got_pose.cpu().numpy().astype(np.float64), d_pose.cpu().numpy().astype(np.float64)) < 1e-5


def test_autotuner_picks_a_candidate_and_caches(tmp_path):
    """gsr_autotune (through the C ABI) times all sixteen candidates on the
    caller's inputs, leaves the fastest in the context, and the Python side
    caches the choice; the tuned context renders the same images."""
    from paper_2411_17660_b300 import autotune as A
    sc = REDUCED["uneven"]()
    params, cams, vm = U.to_device(sc)
    cache = A.TileCache(str(tmp_path / "tiles.json"))
    r = A.tune(params, sc.sh_degree, cams, vm, cache=cache, reps=2)
    assert r["tile"] in A.TILES and r["binning"] in A.BINNINGS and r["batch"] in A.BATCHES
    assert r["fwd_rows"] in A.FWD_ROWS
    assert list(r["ms"]) == list(A.CANDIDATES) and all(t is not None and t > 0 for t in r["ms"].values())
    assert r["ms"][f"{r['tile']}/{r['binning']}/{r['batch']}/{r['fwd_rows']}"] == min(r["ms"].values())
    assert A.tune(params, sc.sh_degree, cams, vm, cache=cache) == r
    tuned = R.GaussianRasterizer(r["tile"], binning=r["binning"], batch=r["batch"], fwd_rows=r["fwd_rows"])
    _assert_same_images_as_default(sc, tuned)


def _assert_same_images_as_default(sc, rast):
    got = U.gpu_forward(sc, rast=rast)[0]
    ref = U.gpu_forward(sc)[0]
    for a, b in zip(got, ref):
        for k in ("color", "depth", "alpha"):
            np.testing.assert_array_equal(a[k], b[k])


def test_autotune_skips_candidates_whose_keys_do_not_fit():
    """A workspace sized for tile 16's keys: the tile-8 candidates report
    GSR_ECAPACITY and are skipped, the others run, and the context keeps the
    fastest of those."""
    from paper_2411_17660_b300 import autotune as A
    sc = REDUCED["window"]()
    params, cams, vm = U.to_device(sc)
    rast = R.GaussianRasterizer(16)
    _, _, _, ws0 = rast.render_forward(params, sc.sh_degree, cams, vm)
    keys16 = rast.info(ws0).keys
    rast8 = R.GaussianRasterizer(8)
    _, _, _, ws8 = rast8.render_forward(params, sc.sh_degree, cams, vm)
    assert rast8.info(ws8).keys > 1.5 * keys16
    ws = rast.alloc_workspace(sc.N, cams, int(keys16 * 1.05) + 3072)
    P = R.pixel_offsets(cams)[-1]
    color = torch.empty(3 * P, device="cuda")
    grads = {k: torch.empty_like(v) for k, v in params.items()}
    g = R.gaussians_struct(*[params[k] for k in R.PARAM_NAMES], sc.sh_degree)
    out = B.Grads(*[grads[k].data_ptr() for k in R.PARAM_NAMES], 0, 0, 0, 0)
    st, entries = rast.ctx.autotune(g, R.view_structs(cams, vm, color), out, ws.data_ptr(), ws.numel(), 1,
                                    torch.cuda.current_stream().cuda_stream)
    assert st == B.OK and len(entries) == len(A.CANDIDATES) == 16
    for e in entries:
        assert (e.status == B.ECAPACITY) == (e.tile == 8), (e.tile, e.binning, e.batch, e.fwd_rows, e.status)
        assert (e.ms > 0) == (e.status == B.OK)
    best = min((e for e in entries if e.status == B.OK), key=lambda e: e.ms)
    # the tuned context renders with its new configuration on a fresh workspace
    color2, _, _, ws2 = rast.render_forward(params, sc.sh_degree, cams, vm)
    assert rast.ctx.get_status(ws2.data_ptr(), ws2.numel(), torch.cuda.current_stream().cuda_stream) == B.OK
    ref = U.gpu_forward(sc)[0]
    for v, c in enumerate(R.split_views(color2, cams, 3)):
        np.testing.assert_array_equal(c.cpu().numpy(), ref[v]["color"])
    assert best.tile in (16, 32)


@pytest.mark.parametrize("deg", [1, 2])
def test_parity_sh_degrees_1_and_2(deg):
    """The degree-1 and degree-2 SH paths (bands cut from the degree-3 scene)."""
    sc = REDUCED["window"]()
    K = (deg + 1) ** 2
    sc = scenes.dataclasses.replace(sc, sh_degree=deg, sh=np.ascontiguousarray(sc.sh[:3 * K]))
    got, state = U.gpu_forward(sc)
    ref = oracle.render(sc)
    for v, (r, g) in enumerate(zip(ref, got)):
        U.compare_images(r, g, f"deg {deg} view {v}")
    gC, gD, gA = U.upstream(sc)
    g = U.gpu_backward(sc, state, gC, gD, gA)
    _, rg = oracle.render_backward(sc, gC, gD, gA)
    U.compare_grads(rg, g, label=f"deg {deg}")


def test_no_gaussians_and_nothing_visible():
    """N = 0, and a scene entirely behind the camera: black images, T = 1,
    zero gradients, zero pose gradients."""
    base = REDUCED["small"]()
    for sc in (base.subset(np.arange(0)), scenes.dataclasses.replace(base, means=base.means * np.array([[1], [1], [-1]], np.float32))):
        got, state = U.gpu_forward(sc)
        for g in got:
            assert np.all(g["color"] == 0) and np.all(g["depth"] == 0) and np.all(g["alpha"] == 0)
        gC, gD, gA = U.upstream(sc)
        gr = U.gpu_backward(sc, state, gC, gD, gA)
        for k in ("means", "log_scales", "quats", "opacity_logits", "sh", "pose"):
            assert np.all(gr[k] == 0), k


def test_many_views_and_tiny_images():
    """64 views (the maximum) of sizes down to 1x1, against the oracle."""
    rng = np.random.default_rng(3)
    sc = REDUCED["window"]()
    cams = []
    for v in range(64):
        H, W = int(rng.integers(1, 40)), int(rng.integers(1, 40))
        c = sc.cameras[v % sc.V]
        cams.append(scenes.Camera(H, W, c.fx * W / 100, c.fy * W / 100, W / 2, H / 2, c.T_cw))
    sc = sc.with_cameras(cams)
    got, state = U.gpu_forward(sc)
    ref = oracle.render(sc)
    for v, (r, g) in enumerate(zip(ref, got)):
        U.compare_images(r, g, f"view {v}")
    gC, gD, gA = U.upstream(sc)
    g = U.gpu_backward(sc, state, gC, gD, gA)
    _, rg = oracle.render_backward(sc, gC, gD, gA)
    U.compare_grads(rg, g, label="64 views")


# ------------------------------------------------------------------ median depth

def _gpu_median(sc, tile=16):
    rast = R.GaussianRasterizer(tile)
    params, cams, vm = U.to_device(sc)
    _, _, _, ws = rast.render_forward(params, sc.sh_degree, cams, vm)
    P = R.pixel_offsets(cams)[-1]
    color = torch.empty(3 * P, device="cuda")
    depth, alpha, med = (torch.empty(P, device="cuda") for _ in range(3))
    rast.forward_raw(params, sc.sh_degree, cams, vm, ws, color, depth, alpha, med)
    torch.cuda.synchronize()
    return rast, params, cams, vm, ws, color, depth, alpha, med


@pytest.mark.parametrize("name", ["window", "uneven", "small"])
def test_median_depth_forward_and_backward(name):
    sc = REDUCED[name]()
    rast, params, cams, vm, ws, color, depth, alpha, med = _gpu_median(sc)
    # rendering the median changes nothing else
    base, _ = U.gpu_forward(sc)
    for v, (b, c, d) in enumerate(zip(base, R.split_views(color, cams, 3), R.split_views(depth, cams))):
        assert np.array_equal(b["color"], c.cpu().numpy().astype(np.float64)), v
        assert np.array_equal(b["depth"], d.cpu().numpy().astype(np.float64)), v
    ref = oracle.render(sc)
    flips = total = 0
    for v, (r, m) in enumerate(zip(ref, R.split_views(med, cams))):
        got = m.cpu().numpy().astype(np.float64)
        err = np.abs(got - r["median_depth"]) / np.maximum(np.abs(r["median_depth"]), 1e-3)
        flip = (r["median_margin"] < U.MARGIN) | U.near_threshold(r)
        bad = err > U.DEPTH_TOL
        assert not (bad & ~flip).any(), f"view {v}: {int((bad & ~flip).sum())} median pixels off"
        flips += int((bad & flip).sum())
        total += bad.size
    assert flips <= U.FLIP_SHARE * total
    # backward: dL/d median depth (with the other upstream gradients)
    gC, gD, gA = U.upstream(sc)
    rng = np.random.default_rng(9)
    gM = [rng.uniform(-1, 1, (c.H, c.W)) for c in sc.cameras]
    flat = lambda arrs: torch.from_numpy(np.concatenate([np.asarray(a, np.float32).reshape(-1) for a in arrs])).cuda()
    grads = {k: torch.empty_like(x) for k, x in params.items()}
    d_pose = torch.empty(len(cams), 6, device="cuda")
    rast.backward_raw(params, sc.sh_degree, cams, vm, ws, flat(gC), flat(gD), flat(gA), grads, d_pose,
                      d_median_depth=flat(gM))
    torch.cuda.synchronize()
    got = {k: x.cpu().numpy().astype(np.float64) for k, x in grads.items()}
    got["pose"] = d_pose.cpu().numpy().astype(np.float64)
    _, rg = oracle.render_backward(sc, gC, gD, gA, gM=gM)
    U.compare_grads(rg, got, label=f"{name} median")


def test_median_gradient_needs_a_median_forward():
    sc = REDUCED["small"]()
    got, state = U.gpu_forward(sc)   # forward without median depth
    rast, params, cams, vm, ws, color, depth, alpha = state
    P = R.pixel_offsets(cams)[-1]
    grads = {k: torch.empty_like(x) for k, x in params.items()}
    with pytest.raises(B.GsrError, match="median"):
        rast.backward_raw(params, sc.sh_degree, cams, vm, ws, None, None, None, grads, None,
                          d_median_depth=torch.zeros(P, device="cuda"))


# ------------------------------------------------------------------ densification statistics

@pytest.mark.parametrize("name", ["window", "uneven", "room"])
def test_densify_stats_against_oracle(name):
    sc = REDUCED[name]()
    _, state = U.gpu_forward(sc)
    rast, params, cams, vm, ws, color, depth, alpha = state
    gC, gD, gA = U.upstream(sc)
    flat = lambda arrs: torch.from_numpy(np.concatenate([np.asarray(a, np.float32).reshape(-1) for a in arrs])).cuda()
    N = sc.N
    grads = {k: torch.empty_like(x) for k, x in params.items()}
    dens = {k: torch.full((N,), np.nan, device="cuda") for k in ("grad", "count", "radius")}
    args = (params, sc.sh_degree, cams, vm, ws, flat(gC), flat(gD), flat(gA), grads, None)
    rast.backward_raw(*args, densify=dens)
    torch.cuda.synchronize()
    got = {k: v.cpu().numpy().astype(np.float64) for k, v in dens.items()}
    _, rg = oracle.render_backward(sc, gC, gD, gA, want_screen=True)
    ref = oracle.densify_stats(sc, rg["screen"])
    sure = ref["margin"] > 1e-3
    assert sure.mean() > 0.99
    np.testing.assert_array_equal(got["count"][sure], ref["count"][sure])
    assert U.rel_l2(got["grad"], ref["grad"]) < U.GRAD_TOL
    m = sure & (ref["count"] > 0)
    np.testing.assert_allclose(got["radius"][m], ref["radius"][m], rtol=1e-4)
    assert not got["radius"][sure & (ref["count"] == 0)].any()
    # accumulate: grad and count add up, the radius keeps its maximum
    rast.backward_raw(*args, accumulate=True, densify=dens)
    torch.cuda.synchronize()
    acc = {k: v.cpu().numpy().astype(np.float64) for k, v in dens.items()}
    np.testing.assert_allclose(acc["grad"], 2 * got["grad"], rtol=1e-6, atol=1e-12)
    np.testing.assert_array_equal(acc["count"], 2 * got["count"])
    np.testing.assert_array_equal(acc["radius"], got["radius"])
