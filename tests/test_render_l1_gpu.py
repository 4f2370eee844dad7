"""GPU tests of gsr_render_l1, the forward render with the L1 loss of Eq.
"rnd_loss" (its L1 colour and depth terms, Sec. 3.3) taken in the forward
blend's epilogue.  It must equal gsr_render followed by gsr_l1_loss: the
images and the loss gradients bit for bit, the loss up to the order of its
FP32 sum.  The stand-alone L1 kernel is pinned to the oracle by the loss
tests, so these comparisons carry that pin over.  Scenes include ragged
image sizes (partial tiles) and median-depth forwards."""
import numpy as np
import pytest
import torch

from paper_2411_17660_b300 import binding as B
from paper_2411_17660_b300 import render as R
from paper_2411_17660_b300 import scenes
from tests import gsr_testutil as U
from tests.test_parity_gpu import REDUCED

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _targets(cams, seed):
    g = torch.Generator(device="cuda").manual_seed(seed)
    P = sum(c.H * c.W for c in cams)
    tc = torch.rand(3 * P, device="cuda", generator=g)
    td = torch.rand(P, device="cuda", generator=g) * 4.0 + 0.5
    return tc, td


def _outputs(P, median):
    nan = lambda n: torch.full((n,), float("nan"), device="cuda")
    return dict(color=nan(3 * P), depth=nan(P), alpha=nan(P), dC=nan(3 * P), dD=nan(P), loss=nan(1),
                med=nan(P) if median else None)


def _both(name, with_depth=True, median=False, depth_out=True, d_depth=True, cw=1.0, dw=0.3, sc=None):
    sc = REDUCED[name]() if sc is None else sc
    params, cams, vm = U.to_device(sc)
    rast = R.GaussianRasterizer(16)
    _, _, _, ws = rast.render_forward(params, sc.sh_degree, cams, vm)
    P = sum(c.H * c.W for c in cams)
    tc, td = _targets(cams, seed=len(name))
    td = td if with_depth else None
    sep, fus = _outputs(P, median), _outputs(P, median)
    rast.forward_raw(params, sc.sh_degree, cams, vm, ws, sep["color"], sep["depth"], sep["alpha"], sep["med"])
    R.l1_loss(rast, cams, vm, sep["color"], sep["depth"], tc, td, cw, dw, sep["dC"],
              sep["dD"] if d_depth else None, sep["loss"])
    rast.forward_l1_raw(params, sc.sh_degree, cams, vm, ws, fus["color"], fus["depth"] if depth_out else None,
                        fus["alpha"], tc, td, cw, dw, fus["dC"], fus["dD"] if d_depth else None, fus["loss"],
                        fus["med"])
    torch.cuda.synchronize()
    assert rast.info(ws).status == B.OK
    return sep, fus, (rast, params, cams, vm, ws, sc)


def _same(a, b):
    np.testing.assert_array_equal(a.cpu().numpy(), b.cpu().numpy())


@pytest.mark.parametrize("name", list(REDUCED))
def test_fused_l1_equals_render_then_l1(name):
    sep, fus, _ = _both(name)
    for k in ("color", "depth", "alpha", "dC", "dD"):
        _same(fus[k], sep[k])
    assert fus["loss"].item() == pytest.approx(sep["loss"].item(), rel=1e-5)
    assert sep["loss"].item() > 0


def test_fused_l1_at_the_benchmark_size():
    """The full 8-view 640x480 window with 100k Gaussians, the benchmark's
    workload and launch configuration (per-tile binning, tile 16)."""
    sep, fus, _ = _both("window", sc=scenes.config_window())
    for k in ("color", "depth", "alpha", "dC", "dD"):
        _same(fus[k], sep[k])
    assert fus["loss"].item() == pytest.approx(sep["loss"].item(), rel=1e-5)


def test_fused_l1_without_depth_target_and_without_depth_outputs():
    sep, fus, _ = _both("uneven", with_depth=False)
    _same(fus["dC"], sep["dC"])
    assert not fus["dD"].abs().any(), "no depth target: zero depth gradient"
    assert fus["loss"].item() == pytest.approx(sep["loss"].item(), rel=1e-5)
    # the depth term uses the composited depth whether or not it is written out
    sep, fus, _ = _both("room", depth_out=False, d_depth=False)
    _same(fus["dC"], sep["dC"])
    assert torch.isnan(fus["depth"]).all()
    assert fus["loss"].item() == pytest.approx(sep["loss"].item(), rel=1e-5)


def test_fused_l1_with_median_depth():
    sep, fus, _ = _both("window", median=True)
    for k in ("color", "depth", "med", "dC", "dD"):
        _same(fus[k], sep[k])
    assert fus["loss"].item() == pytest.approx(sep["loss"].item(), rel=1e-5)


def test_backward_after_the_fused_forward():
    sep, fus, (rast, params, cams, vm, ws, sc) = _both("window")
    out = []
    for o in (sep, fus):
        # the last forward on ws was the fused one; render the separate one again for its backward
        if o is sep:
            rast.forward_raw(params, sc.sh_degree, cams, vm, ws, o["color"], o["depth"], o["alpha"])
        else:
            rast.forward_l1_raw(params, sc.sh_degree, cams, vm, ws, o["color"], o["depth"], o["alpha"],
                                *_targets(cams, seed=len("window")), 1.0, 0.3, o["dC"], o["dD"], o["loss"])
        grads = {k: torch.empty_like(v) for k, v in params.items()}
        d_pose = torch.empty(len(cams), 6, device="cuda")
        rast.backward_raw(params, sc.sh_degree, cams, vm, ws, o["dC"], o["dD"], None, grads, d_pose)
        torch.cuda.synchronize()
        out.append({**{k: v.cpu().numpy() for k, v in grads.items()}, "pose": d_pose.cpu().numpy()})
    for k in out[0]:   # the blend backward's float atomics add in a timing-dependent order
        assert U.rel_l2(out[1][k], out[0][k]) < 1e-5, k


def test_fused_l1_rejects_missing_targets():
    sc = REDUCED["small"]()
    params, cams, vm = U.to_device(sc)
    rast = R.GaussianRasterizer(16)
    _, _, _, ws = rast.render_forward(params, sc.sh_degree, cams, vm)
    P = sum(c.H * c.W for c in cams)
    color = torch.empty(3 * P, device="cuda")
    g = R.gaussians_struct(*[params[k] for k in R.PARAM_NAMES], sc.sh_degree)
    views = R.view_structs(cams, vm, color, None, None)
    loss = torch.empty(1, device="cuda")
    st = rast.ctx.render_l1(g, views, [B.L1View(0, 0, color.data_ptr(), 0)] * len(cams), 1.0, 0.0,
                            loss.data_ptr(), ws.data_ptr(), ws.numel(), 0)
    assert st == B.EINVAL
    st = rast.ctx.render_l1(g, views, [B.L1View(color.data_ptr(), 0, color.data_ptr(), 0)] * len(cams), 1.0, 0.0,
                            0, ws.data_ptr(), ws.numel(), 0)
    assert st == B.EINVAL
