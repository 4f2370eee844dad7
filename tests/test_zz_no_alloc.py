"""gsr_render_noalloc: the forward render for callers that cannot allocate.

Plug-ins that run inside another framework's execution phase (where only that
framework owns the device allocator) and real-time loops that must not
allocate cannot provide gsr_render's workspace.  gsr_render_noalloc renders
into a static device array inside the library instead.  These tests call it
through the C ABI and require the same images as gsr_render on the same
inputs, on two calls in a row (the second on a different scene, so leftovers
of the first call in the shared array must not matter), and a clear rejection
of a scene whose workspace cannot fit the static array.

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
    for a, b in ((c2, color), (d2, depth), (a2, alpha)):
        np.testing.assert_allclose(a.cpu().numpy(), b.cpu().numpy(), rtol=0, atol=U.COLOR_TOL)


def test_noalloc_matches_render_on_two_calls():
    rast = R.GaussianRasterizer(16)
    _render_both(rast, scenes.config_window(N=5000, V=4, H=75, W=100, f=78.0))
    _render_both(rast, scenes.config_room(N=20000, H=140, W=250, f=125.0))


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
