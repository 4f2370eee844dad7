"""GPU parity of the density-control kernels (csrc/density.cu) against the
FP64 oracle (oracle/density.py), through the C ABI.

Every decision is compared exactly (which Gaussians are pruned, cloned,
split; which live Gaussian each dead slot draws, checked through the copied
parameters bit for bit); computed parameters (split children, relocated
opacities and scales, noise steps) within FP32 rounding.  Sizes span several
4096-value scan blocks with a ragged tail, plus a 2M-Gaussian case on the
decisions."""
import math

import numpy as np
import pytest
import torch

from oracle import density as OD
from paper_2411_17660_b300 import binding as B
from paper_2411_17660_b300 import render as R
from paper_2411_17660_b300.density import DensityControl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _scene(N, deg=3, seed=0):
    rng = np.random.default_rng(seed)
    C = 3 * (deg + 1) ** 2
    g = OD.Gaussians(means=rng.normal(0, 2, (3, N)).astype(np.float32),
                     log_scales=rng.normal(-4, 0.8, (3, N)).astype(np.float32),
                     quats=rng.normal(0, 1, (4, N)).astype(np.float32),
                     opacity_logits=rng.normal(-1, 3, N).astype(np.float32),
                     sh=rng.normal(0, 0.3, (C, N)).astype(np.float32))
    count = rng.integers(0, 9, N).astype(np.float32)
    grad = (count * rng.exponential(2e-4, N)).astype(np.float32)
    radius = rng.uniform(0, 40, N).astype(np.float32)
    return g, grad, count, radius


def _dev(g: OD.Gaussians):
    return {k: torch.from_numpy(np.ascontiguousarray(getattr(g, k))).cuda() for k in R.PARAM_NAMES}


def _host(d):
    return OD.Gaussians(*(d[k].cpu().numpy().astype(np.float64) for k in R.PARAM_NAMES))


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


ADC = dict(grad_threshold=2e-4, split_scale=0.02, min_opacity=0.005, max_screen_radius=30.0, max_world_scale=0.1)


@pytest.mark.parametrize("N", [1, 4095, 4096 * 3 + 17])
def test_adc_matches_oracle(N):
    g, grad, count, radius = _scene(N, seed=N)
    normals = np.random.default_rng(N + 1).normal(0, 1, (2, 3, N)).astype(np.float32)
    dc = DensityControl(R.GaussianRasterizer(16))
    out, n = dc.densify_adc(_dev(g), 3, _t(grad), _t(count), _t(radius), _t(normals), **ADC)
    ref = OD.adc(g, grad, count, radius, normals, **ADC)
    assert int(n.item()) == ref.N
    got = _host(out)
    d = OD.adc_decisions(g, grad, count, radius, **ADC)
    split_rows = np.repeat(d["split"][~d["pruned"]], np.where(d["clone"] | d["split"], 2, 1)[~d["pruned"]])
    for k in R.PARAM_NAMES:
        a, b = getattr(got, k), getattr(ref, k)
        assert a.shape == b.shape, k
        if k in ("means", "log_scales"):
            np.testing.assert_array_equal(a[..., ~split_rows], b[..., ~split_rows])   # exact copies
            np.testing.assert_allclose(a[..., split_rows], b[..., split_rows], rtol=2e-6, atol=2e-7)
        else:
            np.testing.assert_array_equal(a, b)


def _around(rng, t, n):
    """n floats within one unit in the last place of the double t."""
    c = np.float32(t)
    k = rng.integers(-1, 2, n)
    lo, hi = np.nextafter(c, np.float32(-np.inf)), np.nextafter(c, np.float32(np.inf))
    return np.where(k < 0, lo, np.where(k > 0, hi, c)).astype(np.float32)


def test_adc_decisions_at_the_thresholds():
    """Inputs one float apart around every threshold (the density test's
    grad = threshold x count, ln split_scale, logit(min_opacity),
    ln max_world_scale): the kernel's FP32 compares must take the decisions of
    the oracle's FP64 ones."""
    N = 3 * 4096 + 5
    rng = np.random.default_rng(77)
    g, _, _, radius = _scene(N, seed=77)
    radius[:] = 0.0
    count = rng.integers(1, 9, N).astype(np.float32)
    thr = float(np.float32(ADC["grad_threshold"]))
    grad = _around(rng, 0.0, N)
    for c in range(1, 9):   # the product is exact in FP64; its neighbours in FP32
        sel = count == c
        grad[sel] = _around(rng, thr * c, int(sel.sum()))
    ls_split = math.log(float(np.float32(ADC["split_scale"])))
    ls_world = math.log(float(np.float32(ADC["max_world_scale"])))
    g.log_scales[0] = _around(rng, ls_split, N)
    g.log_scales[0, 1::4] = _around(rng, ls_world, len(range(1, N, 4)))
    g.log_scales[1:] = g.log_scales[0] - 1.0
    mo = float(np.float32(ADC["min_opacity"]))
    g.opacity_logits[:] = _around(rng, math.log(mo / (1.0 - mo)), N)
    g.opacity_logits[::2] = 2.0   # opaque: the split and clone branches too
    normals = rng.normal(0, 1, (2, 3, N)).astype(np.float32)
    dc = DensityControl(R.GaussianRasterizer(16))
    out, n = dc.densify_adc(_dev(g), 3, _t(grad), _t(count), _t(radius), _t(normals), **ADC)
    d = OD.adc_decisions(g, grad, count, radius, **ADC)
    for k in ("dense", "big", "pruned"):   # every branch is taken on both sides of its threshold
        assert 0 < int(d[k].sum()) < N, k
    assert int(n.item()) == int(d["n_out"].sum())
    ref = OD.adc(g, grad, count, radius, normals, **ADC)
    got = _host(out)
    split_rows = np.repeat(d["split"][~d["pruned"]], np.where(d["clone"] | d["split"], 2, 1)[~d["pruned"]])
    for k in R.PARAM_NAMES:
        a, b = getattr(got, k), getattr(ref, k)
        assert a.shape == b.shape, k
        if k in ("means", "log_scales"):
            np.testing.assert_array_equal(a[..., ~split_rows], b[..., ~split_rows])
            np.testing.assert_allclose(a[..., split_rows], b[..., split_rows], rtol=2e-6, atol=2e-7)
        else:
            np.testing.assert_array_equal(a, b)


def test_adc_truncates_at_capacity_and_reports_the_count():
    g, grad, count, radius = _scene(5000, seed=3)
    normals = np.zeros((2, 3, 5000), np.float32)
    dc = DensityControl(R.GaussianRasterizer(16))
    full, n = dc.densify_adc(_dev(g), 3, _t(grad), _t(count), _t(radius), _t(normals), **ADC)
    cut, n2 = dc.densify_adc(_dev(g), 3, _t(grad), _t(count), _t(radius), _t(normals), capacity=1000, **ADC)
    assert int(n2.item()) == int(n.item()) > 1000
    for k in R.PARAM_NAMES:
        np.testing.assert_array_equal(cut[k].cpu().numpy(), full[k].cpu().numpy()[..., :1000])


def test_adc_with_nothing_to_do_and_with_everything_pruned():
    g, grad, count, radius = _scene(300, seed=4)
    dc = DensityControl(R.GaussianRasterizer(16))
    zero = np.zeros(300, np.float32)
    out, n = dc.densify_adc(_dev(g), 3, _t(zero), _t(zero), _t(zero), _t(np.zeros((2, 3, 300), np.float32)),
                            grad_threshold=1.0, split_scale=1.0, min_opacity=1e-9)
    assert int(n.item()) == 300
    np.testing.assert_array_equal(out["sh"].cpu().numpy(), g.sh)
    out, n = dc.densify_adc(_dev(g), 3, _t(zero), _t(zero), _t(zero), _t(np.zeros((2, 3, 300), np.float32)),
                            grad_threshold=1.0, split_scale=1.0, min_opacity=0.999999)
    assert int(n.item()) == 0 and out["means"].shape == (3, 0)


@pytest.mark.parametrize("N,deg", [(4096 * 2 + 5, 3), (777, 0)])
def test_relocate_matches_oracle(N, deg):
    g, _, _, _ = _scene(N, deg=deg, seed=10 + N)
    draws = np.random.default_rng(N).integers(0, 1 << 32, N, dtype=np.uint64).astype(np.uint32)
    dc = DensityControl(R.GaussianRasterizer(16))
    out, moved = dc.mcmc_relocate(_dev(g), deg, _t(draws.view(np.int32)), 0.005)
    ref, src = OD.mcmc_relocate(g, draws.astype(np.uint64), 0.005)
    got = _host(out)
    assert int(moved.item()) == int((src >= 0).sum())
    # the copied parameters are bit-exact, so they check every draw
    for k in ("means", "quats", "sh"):
        np.testing.assert_array_equal(getattr(got, k), getattr(ref, k))
    np.testing.assert_allclose(got.opacity_logits, ref.opacity_logits, rtol=1e-5, atol=2e-5)
    np.testing.assert_allclose(got.log_scales, ref.log_scales, rtol=1e-6, atol=2e-6)


def test_relocate_without_live_gaussians_copies_the_input():
    g, _, _, _ = _scene(500, seed=20)
    g.opacity_logits[:] = -12.0
    draws = np.arange(500, dtype=np.uint32) * 7919
    dc = DensityControl(R.GaussianRasterizer(16))
    out, moved = dc.mcmc_relocate(_dev(g), 3, _t(draws.view(np.int32)), 0.005)
    assert int(moved.item()) == 0
    for k in R.PARAM_NAMES:
        np.testing.assert_array_equal(out[k].cpu().numpy(), getattr(g, k))


def test_relocate_draws_at_two_million():
    N = 2_000_000
    rng = np.random.default_rng(5)
    lg = rng.normal(-3, 2.5, N).astype(np.float32)
    g = OD.Gaussians(means=np.zeros((3, N), np.float32) + np.arange(N, dtype=np.float32),
                     log_scales=np.full((3, N), -4, np.float32), quats=np.tile(np.array([[1], [0], [0], [0]],
                                                                                       np.float32), (1, N)),
                     opacity_logits=lg, sh=np.zeros((3, N), np.float32))
    draws = rng.integers(0, 1 << 32, N, dtype=np.uint64).astype(np.uint32)
    dc = DensityControl(R.GaussianRasterizer(16))
    out, moved = dc.mcmc_relocate(_dev(g), 0, _t(draws.view(np.int32)), 0.005)
    dead, src, drawn = OD.relocate_sources(lg, draws.astype(np.uint64), 0.005)
    assert int(moved.item()) == int(dead.sum())
    # means hold each Gaussian's index, so the copied means name the source
    got_src = out["means"][0].cpu().numpy().astype(np.int64)
    want = np.where(src >= 0, src, np.arange(N))
    assert np.array_equal(got_src, want)


def test_adc_decisions_at_two_million():
    N = 2_000_000
    g, grad, count, radius = _scene(N, deg=0, seed=6)
    dc = DensityControl(R.GaussianRasterizer(16))
    out, n = dc.densify_adc(_dev(g), 0, _t(grad), _t(count), _t(radius), _t(np.zeros((2, 3, N), np.float32)),
                            sync=False, **ADC)
    d = OD.adc_decisions(g, grad, count, radius, **ADC)
    assert int(n.item()) == int(d["n_out"].sum())
    keep = ~d["pruned"]
    reps = np.where(d["clone"] | d["split"], 2, 1)[keep]
    want_logit = np.repeat(g.opacity_logits[keep], reps)
    np.testing.assert_array_equal(out["opacity_logits"][: want_logit.size].cpu().numpy(), want_logit)


def test_noise_matches_oracle():
    g, _, _, _ = _scene(4096 + 333, seed=30)
    g.opacity_logits[:50] = np.float32(math.log(0.005 / 0.995))
    eta = np.random.default_rng(31).normal(0, 1, (3, g.N)).astype(np.float32)
    dc = DensityControl(R.GaussianRasterizer(16))
    params = _dev(g)
    new = dc.mcmc_noise(params, 3, _t(eta), 5e3).cpu().numpy().astype(np.float64)
    ref = OD.mcmc_noise(g, eta, 5e3)
    step_ref = ref - g.means.astype(np.float64)
    step = new - g.means.astype(np.float64)
    err = np.abs(step - step_ref)
    # FP32 error of Sigma eta = M (M^T eta): relative to |M|^2 |eta|, not to the
    # (possibly cancelled) step; plus the rounding of mean + step
    o = OD.sigmoid(g.opacity_logits)
    gate = OD.sigmoid(-100.0 * (o - 0.005))
    smax2 = np.exp(2.0 * g.log_scales.astype(np.float64)).max(axis=0)
    bound = 1e-5 * 5e3 * gate * smax2 * np.linalg.norm(eta, axis=0) + 4e-7 * (1 + np.abs(g.means))
    assert np.all(err <= bound), float(np.max(err / bound))
    # in place gives the same
    dc.mcmc_noise(params, 3, _t(eta), 5e3, means_out=params["means"])
    np.testing.assert_array_equal(params["means"].cpu().numpy(), new.astype(np.float32))


def test_density_calls_reject_bad_arguments():
    g, grad, count, radius = _scene(100, seed=40)
    dc = DensityControl(R.GaussianRasterizer(16))
    params = _dev(g)
    gs = R.gaussians_struct(*[params[k] for k in R.PARAM_NAMES], 3)
    ws = torch.empty(dc.ctx.density_workspace_size(100), dtype=torch.uint8, device="cuda")
    alias = B.GaussiansOut(100, *[params[k].data_ptr() for k in R.PARAM_NAMES])
    n = torch.zeros(1, dtype=torch.int32, device="cuda")
    draws = torch.zeros(100, dtype=torch.int32, device="cuda")
    st = dc.ctx.mcmc_relocate(gs, draws.data_ptr(), 0.005, alias, n.data_ptr(), ws.data_ptr(), ws.numel(), 0)
    assert st == B.EINVAL
    out, s = dc._outputs(params, 50)
    st = dc.ctx.mcmc_relocate(gs, draws.data_ptr(), 0.005, s, n.data_ptr(), ws.data_ptr(), ws.numel(), 0)
    assert st == B.EINVAL   # room for 50 < N
    prm = B.AdcParams(2e-4, 0.02, 1.5, 0.0, 0.0)   # min_opacity out of range
    out, s = dc._outputs(params, 200)
    st = dc.ctx.densify_adc(gs, _t(grad).data_ptr(), _t(count).data_ptr(), 0, _t(np.zeros((2, 3, 100), np.float32)).data_ptr(),
                            prm, s, n.data_ptr(), ws.data_ptr(), ws.numel(), 0)
    assert st == B.EINVAL
    st = dc.ctx.densify_adc(gs, 0, 0, 0, 0, B.AdcParams(2e-4, 0.02, 0.005, 0.0, 0.0), s, n.data_ptr(),
                            ws.data_ptr(), 16, 0)
    assert st == B.EINVAL   # workspace too small (and missing statistics)
