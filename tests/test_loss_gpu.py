"""GPU parity of the mixed L1 + SSIM + depth loss of Eq. "rnd_loss" (Sec. 3.3)
against the FP64 oracle (oracle/loss.py), through the C ABI.

The loss is checked to 1e-5 relative and its image gradients to 1e-3 relative
L2 (the gradient tolerance of the renderer), on rendered images of the
reduced window scene and on random images of ragged sizes that are not
multiples of the kernel's 32x32 tile."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle.loss as OL
from paper_2411_17660_b300 import render as R
from paper_2411_17660_b300 import scenes

from tests import gsr_testutil as U

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")

LOSS_REL = 1e-5


def _flat(arrs):
    return torch.from_numpy(np.concatenate([np.asarray(a, np.float32).reshape(-1) for a in arrs])).cuda()


def _run(cams, colors, depths, tcolors, tdepths, lambda1, lambda2, rast=None):
    rast = rast or R.GaussianRasterizer(16)
    V = len(cams)
    vm = torch.zeros(V, 3, 4, device="cuda")
    vm[:, :, :3] = torch.eye(3, device="cuda")
    color, depth, tc = _flat(colors), _flat(depths), _flat(tcolors)
    td = None if tdepths is None else _flat(tdepths)
    dC, dD = torch.full_like(color, np.nan), torch.full_like(depth, np.nan)
    loss = torch.full((1,), np.nan, device="cuda")
    R.rgbd_loss(rast, cams, vm, color, depth, tc, td, lambda1, lambda2, dC, dD, loss)
    torch.cuda.synchronize()
    return loss.item(), R.split_views(dC, cams, 3), R.split_views(dD, cams)


def _check(cams, colors, depths, tcolors, tdepths, lambda1, lambda2):
    loss, dC, dD = _run(cams, colors, depths, tcolors, tdepths, lambda1, lambda2)
    c64 = [np.asarray(c, np.float32).astype(np.float64) for c in colors]
    d64 = [np.asarray(d, np.float32).astype(np.float64) for d in depths]
    t64 = [np.asarray(c, np.float32).astype(np.float64) for c in tcolors]
    td64 = [None] * len(cams) if tdepths is None else [np.asarray(d, np.float32).astype(np.float64)
                                                         for d in tdepths]
    ref, rC, rD = OL.window_loss_and_grads(c64, t64, d64, td64, lambda1, lambda2)
    assert loss == pytest.approx(ref, rel=LOSS_REL)
    gC = np.concatenate([g.cpu().numpy().reshape(-1) for g in dC]).astype(np.float64)
    gD = np.concatenate([g.cpu().numpy().reshape(-1) for g in dD]).astype(np.float64)
    eC = np.concatenate([g.reshape(-1) for g in rC])
    eD = np.concatenate([g.reshape(-1) for g in rD])
    assert np.isfinite(gC).all() and np.isfinite(gD).all()
    assert U.rel_l2(gC, eC) < U.GRAD_TOL
    if tdepths is None:
        assert not gD.any()
    else:
        # the depth gradient is (1 - lambda1) sign(d) / P: exact up to rounding
        np.testing.assert_allclose(gD, eD, rtol=1e-6, atol=1e-12)
    return loss, ref


def test_rgbd_loss_on_rendered_window():
    sc = scenes.config_window(N=5000, V=4, H=75, W=100, f=78.0)
    views, _ = U.gpu_forward(sc)
    cams = [R.Intrinsics(c.H, c.W, float(c.fx), float(c.fy), float(c.cx), float(c.cy)) for c in sc.cameras]
    _check(cams, [v["color"] for v in views], [v["depth"] for v in views], sc.target_color, sc.target_depth,
           0.8, 0.2)


@pytest.mark.parametrize("lambda1,lambda2,with_depth", [(0.9, 0.2, True), (0.8, 0.2, False), (1.0, 1.0, True)])
def test_rgbd_loss_ragged_sizes(lambda1, lambda2, with_depth):
    rng = np.random.default_rng(11)
    sizes = [(37, 45), (1, 1), (64, 32), (33, 97), (5, 3)]
    cams = [R.Intrinsics(H, W, 100.0, 100.0, W / 2, H / 2) for H, W in sizes]
    base = [rng.uniform(0, 1, (3, H, W)) for H, W in sizes]
    colors = [np.clip(b + rng.normal(0, 0.1, b.shape), 0, 1) for b in base]
    depths = [rng.uniform(1, 4, (H, W)) for H, W in sizes]
    tdepths = [d + rng.normal(0, 0.05, d.shape) for d in depths] if with_depth else None
    _check(cams, colors, depths, base, tdepths, lambda1, lambda2)


def test_rgbd_loss_of_identical_images_is_zero():
    rng = np.random.default_rng(3)
    sizes = [(40, 50), (31, 17)]
    cams = [R.Intrinsics(H, W, 100.0, 100.0, W / 2, H / 2) for H, W in sizes]
    img = [rng.uniform(0, 1, (3, H, W)) for H, W in sizes]
    dep = [rng.uniform(1, 4, (H, W)) for H, W in sizes]
    loss, dC, dD = _run(cams, img, dep, img, dep, 0.9, 0.2)
    # SSIM of an image with itself is 1 and every L1 term is 0
    assert abs(loss) < 1e-5
    for g in dC:
        assert g.abs().max().item() < 1e-6
    for g in dD:
        assert not g.any()


def test_rgbd_loss_without_ssim_equals_l1_front_end():
    rng = np.random.default_rng(4)
    sizes = [(48, 64), (30, 41)]
    cams = [R.Intrinsics(H, W, 100.0, 100.0, W / 2, H / 2) for H, W in sizes]
    colors = [rng.uniform(0, 1, (3, H, W)) for H, W in sizes]
    tcol = [rng.uniform(0, 1, (3, H, W)) for H, W in sizes]
    depths = [rng.uniform(1, 4, (H, W)) for H, W in sizes]
    tdep = [rng.uniform(1, 4, (H, W)) for H, W in sizes]
    rast = R.GaussianRasterizer(16)
    loss, dC, dD = _run(cams, colors, depths, tcol, tdep, 0.7, 0.0, rast)
    vm = torch.zeros(len(cams), 3, 4, device="cuda")
    vm[:, :, :3] = torch.eye(3, device="cuda")
    color, depth = _flat(colors), _flat(depths)
    eC, eD, el = torch.empty_like(color), torch.empty_like(depth), torch.empty(1, device="cuda")
    R.l1_loss(rast, cams, vm, color, depth, _flat(tcol), _flat(tdep), 0.7, 0.3, eC, eD, el)
    torch.cuda.synchronize()
    assert loss == pytest.approx(el.item(), rel=1e-5)
    np.testing.assert_allclose(torch.cat([g.reshape(-1) for g in dC]).cpu().numpy(), eC.cpu().numpy(),
                               rtol=1e-6, atol=1e-12)
    np.testing.assert_allclose(torch.cat([g.reshape(-1) for g in dD]).cpu().numpy(), eD.cpu().numpy(),
                               rtol=1e-6, atol=1e-12)


def test_rgbd_loss_rejects_bad_weights():
    cams = [R.Intrinsics(8, 8, 10.0, 10.0, 4.0, 4.0)]
    with pytest.raises(Exception, match="lambda"):
        _run(cams, [np.zeros((3, 8, 8))], [np.ones((8, 8))], [np.zeros((3, 8, 8))], None, 1.5, 0.2)
