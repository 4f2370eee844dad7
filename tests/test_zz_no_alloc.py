"""gsr_render_noalloc: the forward render for callers that cannot allocate.

Plug-ins that run inside another framework's execution phase (where only that
framework owns the device allocator) and real-time loops that must not
allocate cannot provide gsr_render's workspace.  gsr_render_noalloc renders
into a static device array inside the library instead.  These tests call it
through the C ABI and require the same images as gsr_render on the same
inputs, bit for bit, on two calls in a row (the second on a different scene,
so leftovers of the first call in the shared array must not matter), report
in the status they write when the tile keys overflow the array, and reject
clearly a scene whose workspace cannot fit it at all.

This file is collected last on purpose: a failure here leaves every other
test already run.
"""
import numpy as np
import pytest
import torch

from paper_2411_17660_b300 import binding as B
from paper_2411_17660_b300 import render as R
from paper_2411_17660_b300 import scenes
from tests import gsr_testutil as U

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _render_both(rast, sc):
    params, cams, vm = U.to_device(sc)
    color, depth, alpha, _ = rast.render_forward(params, sc.sh_degree, cams, vm)   # gsr_render
    c2, d2, a2 = torch.full_like(color, -1.0), torch.full_like(depth, -1.0), torch.full_like(alpha, -1.0)
    status = torch.full((1,), -99, dtype=torch.int32, device="cuda")
    g = R.gaussians_struct(*[params[k] for k in R.PARAM_NAMES], sc.sh_degree)
    views = R.view_structs(cams, vm, c2, d2, a2)
    st = rast.ctx.render_noalloc(g, views, status.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert st == B.OK, rast.ctx.lib.gsr_last_error(rast.ctx.h).decode()
    torch.cuda.synchronize()
    assert status.item() == 0
    # the same kernels on the same inputs: bit-identical images
    for a, b in ((c2, color), (d2, depth), (a2, alpha)):
        np.testing.assert_array_equal(a.cpu().numpy(), b.cpu().numpy())


def test_noalloc_matches_render_on_two_calls():
    rast = R.GaussianRasterizer(16)
    _render_both(rast, scenes.config_window(N=5000, V=4, H=75, W=100, f=78.0))
    _render_both(rast, scenes.config_room(N=20000, H=140, W=250, f=125.0))


def test_noalloc_reports_key_overflow_in_its_status():
    """A scene whose smallest workspace fits in the static array but whose
    tile keys do not (8,000 wide Gaussians over a 512x512 view, about 5M
    keys against room for about 2.7M): the call itself succeeds and the
    device status it writes is GSR_ECAPACITY; a render of a small scene right
    after it is correct again."""
    import dataclasses
    base = scenes.config_small(N=8000, H=512, W=512, f=150.0)
    rng = np.random.default_rng(3)
    sc = dataclasses.replace(base, log_scales=np.full((3, 8000), np.log(2.0), np.float32),
                             opacity_logits=np.ascontiguousarray(rng.normal(0.0, 0.3, 8000).astype(np.float32)))
    params, cams, vm = U.to_device(sc)
    P = sum(c.H * c.W for c in cams)
    out = [torch.empty(3 * P, device="cuda"), torch.empty(P, device="cuda"), torch.empty(P, device="cuda")]
    status = torch.full((1,), -99, dtype=torch.int32, device="cuda")
    rast = R.GaussianRasterizer(16)
    g = R.gaussians_struct(*[params[k] for k in R.PARAM_NAMES], sc.sh_degree)
    st = rast.ctx.render_noalloc(g, R.view_structs(cams, vm, *out), status.data_ptr(),
                                 torch.cuda.current_stream().cuda_stream)
    assert st == B.OK, rast.ctx.lib.gsr_last_error(rast.ctx.h).decode()
    torch.cuda.synchronize()
    assert status.item() == B.ECAPACITY
    _render_both(rast, scenes.config_window(N=5000, V=4, H=75, W=100, f=78.0))


def test_noalloc_rejects_scene_larger_than_static_scratch():
    sc = scenes.config_small(N=64)
    params, _, _ = U.to_device(sc)
    rast = R.GaussianRasterizer(16)
    big = [R.Intrinsics(8192, 8192, 4000.0, 4000.0, 4096.0, 4096.0)]   # 64M pixels of per-pixel state
    vm = torch.tensor([[[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 1, 0]]], dtype=torch.float32, device="cuda")
    out = torch.empty(3 * 8192 * 8192, device="cuda")
    g = R.gaussians_struct(*[params[k] for k in R.PARAM_NAMES], sc.sh_degree)
    st = rast.ctx.render_noalloc(g, R.view_structs(big, vm, out), 0, torch.cuda.current_stream().cuda_stream)
    assert st == B.EINVAL
    assert "static scratch" in rast.ctx.lib.gsr_last_error(rast.ctx.h).decode()
