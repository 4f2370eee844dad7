"""GPU parity of the surfel (2DGS) renderer against the FP64 surfel oracle
(oracle/surfel.py), through the C ABI: colour, depth, opacity, normal map and
depth distortion, and every gradient including the poses."""
import numpy as np
import pytest
import torch

from oracle import surfel as OS
from paper_2411_17660_b300 import render as R
from paper_2411_17660_b300 import scenes
from tests import gsr_testutil as U

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def surfel_scene(name="window"):
    if name == "window":
        return scenes.config_window(N=900, V=3, H=48, W=64, f=52.0)
    if name == "room":
        return scenes.config_room(N=700, H=56, W=90, f=45.0)
    return scenes.config_uneven(N=1200, V=3, res_scale=0.08)


def gpu_surfels(sc, tile=16, binning="tile"):
    rast = R.GaussianRasterizer(tile, binning=binning)
    params, cams, vm = U.to_device(sc)
    P = R.pixel_offsets(cams)[-1]
    ws = rast.alloc_workspace(sc.N, cams, 1 << 20)
    out = dict(color=torch.empty(3 * P, device="cuda"), depth=torch.empty(P, device="cuda"),
               alpha=torch.empty(P, device="cuda"), normal=torch.empty(3 * P, device="cuda"),
               distortion=torch.empty(P, device="cuda"))
    rast.surfels_forward_raw(params, sc.sh_degree, cams, vm, ws, out["color"], out["depth"], out["alpha"],
                             out["normal"], out["distortion"])
    torch.cuda.synchronize()
    info = rast.info(ws)
    assert info.status == 0, info.status
    views = []
    for v in range(len(cams)):
        d = {}
        for k, ch in (("color", 3), ("depth", 1), ("alpha", 1), ("normal", 3), ("distortion", 1)):
            d[k] = R.split_views(out[k], cams, ch)[v].cpu().numpy().astype(np.float64)
        views.append(d)
    return views, (rast, params, cams, vm, ws)


def compare_surfels(ref, got, label):
    flip = ref["margin"] < U.SURFEL_MARGIN
    err_c = np.abs(got["color"] - ref["color"]).max(0)
    err_n = np.abs(got["normal"] - ref["normal"]).max(0)
    err_a = np.abs(got["alpha"] - ref["alpha"])
    err_d = np.abs(got["depth"] - ref["depth"]) / np.maximum(np.abs(ref["depth"]), 1e-3)
    err_l = np.abs(got["distortion"] - ref["distortion"]) / np.maximum(np.abs(ref["distortion"]), 1e-3)
    bad = (err_c > U.COLOR_TOL) | (err_n > U.COLOR_TOL) | (err_a > U.ALPHA_TOL) | (err_d > U.DEPTH_TOL) | \
        (err_l > 1e-3)
    hard = bad & ~flip
    where = [(int(x), int(y), float(got["depth"][y, x]), float(ref["depth"][y, x]), float(ref["margin"][y, x]))
             for y, x in zip(*np.nonzero(hard))][:4]
    assert not hard.any(), (f"{label}: {int(hard.sum())} pixels off at {where}; worst colour {err_c[~flip].max():.3g} "
                            f"normal {err_n[~flip].max():.3g} alpha {err_a[~flip].max():.3g} "
                            f"depth {err_d[~flip].max():.3g} distortion {err_l[~flip].max():.3g}")
    return int((bad & flip).sum()), bad.size


@pytest.mark.parametrize("name", ["window", "room", "uneven"])
def test_surfel_forward_parity(name):
    sc = surfel_scene(name)
    got, _ = gpu_surfels(sc)
    ref = OS.render_surfels(sc)
    flips = total = 0
    for v, (r, g) in enumerate(zip(ref, got)):
        f, t = compare_surfels(r, g, f"{name} view {v}")
        flips += f
        total += t
        assert (r["alpha"] > 0).mean() > 0.05
    assert flips <= U.FLIP_SHARE * total


def test_surfel_tile_size_invariance():
    sc = surfel_scene("window")
    base, _ = gpu_surfels(sc, 16)
    for tile in (8, 32):
        other, _ = gpu_surfels(sc, tile)
        for a, b in zip(base, other):
            for k in a:
                assert np.array_equal(a[k], b[k]), (tile, k)


@pytest.mark.parametrize("name", ["window", "room", "uneven"])
def test_surfel_backward_parity(name):
    sc = surfel_scene(name)
    _, (rast, params, cams, vm, ws) = gpu_surfels(sc)
    rng = np.random.default_rng(17)
    up = {k: [rng.uniform(-1, 1, (ch, c.H, c.W)) if ch > 1 else rng.uniform(-1, 1, (c.H, c.W))
              for c in sc.cameras] for k, ch in (("color", 3), ("depth", 1), ("alpha", 1), ("normal", 3),
                                                 ("distortion", 1))}
    flat = lambda arrs: torch.from_numpy(np.concatenate([np.asarray(a, np.float32).reshape(-1) for a in arrs])).cuda()
    grads = {k: torch.empty_like(x) for k, x in params.items()}
    d_pose = torch.empty(len(cams), 6, device="cuda")
    rast.surfels_backward_raw(params, sc.sh_degree, cams, vm, ws, flat(up["color"]), flat(up["depth"]),
                              flat(up["alpha"]), flat(up["normal"]), flat(up["distortion"]), grads, d_pose)
    torch.cuda.synchronize()
    got = {k: v.cpu().numpy().astype(np.float64) for k, v in grads.items()}
    got["pose"] = d_pose.cpu().numpy().astype(np.float64)
    _, ref = OS.render_surfels_backward(sc, up["color"], up["depth"], up["alpha"], up["normal"], up["distortion"])
    assert not got["log_scales"][2].any()
    U.compare_grads(ref, got, label=f"{name} surfels")


def test_surfel_backward_needs_a_surfel_forward():
    from paper_2411_17660_b300 import binding as B
    sc = surfel_scene("window")
    _, state = U.gpu_forward(sc)   # a 3-D Gaussian forward on this workspace
    rast, params, cams, vm, ws = state[:5]
    grads = {k: torch.empty_like(x) for k, x in params.items()}
    with pytest.raises(B.GsrError, match="surfel"):
        rast.surfels_backward_raw(params, sc.sh_degree, cams, vm, ws, None, None, None, None, None, grads, None)
