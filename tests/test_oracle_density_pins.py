"""Pins of the density-control oracle (oracle/density.py) against facts that
do not come from it: library routines (math.exp, scipy rotations and
quadrature), closed forms of the relocation rule, and hand-built cases of
every adaptive-density-control branch."""
import math

import numpy as np
import pytest
from scipy import integrate
from scipy.spatial.transform import Rotation

from oracle import density as D


def _gaussians(N, seed=0, C=3):
    rng = np.random.default_rng(seed)
    return D.Gaussians(means=rng.normal(0, 1, (3, N)).astype(np.float32),
                       log_scales=rng.normal(-3, 0.5, (3, N)).astype(np.float32),
                       quats=rng.normal(0, 1, (4, N)).astype(np.float32),
                       opacity_logits=rng.normal(0, 2, N).astype(np.float32),
                       sh=rng.normal(0, 1, (C, N)).astype(np.float32))


# ---------------------------------------------------------------- the FP32 sigmoid of the sampling weights
def test_exp32_is_within_one_ulp_of_exp():
    x = np.linspace(-87, 88, 400001).astype(np.float32)
    e = D.exp32(x).astype(np.float64)
    r = np.exp(x.astype(np.float64))
    assert np.max(np.abs(e - r) / r) < 2.0 ** -23


def test_sigmoid32_matches_the_logistic_function():
    x = np.linspace(-30, 30, 10001).astype(np.float32)
    s = D.sigmoid32(x).astype(np.float64)
    ref = np.array([1.0 / (1.0 + math.exp(-float(v))) for v in x])
    assert np.max(np.abs(s - ref) / ref) < 3 * 2.0 ** -24
    assert D.sigmoid32(np.float32(0.0)) == np.float32(0.5)


def test_weights_are_proportional_to_opacity_and_zero_for_dead():
    lg = np.array([-10.0, -5.3, 0.0, 4.0], np.float32)   # sigma 4.5e-5, 5.0e-3, 0.5, 0.982
    dead, w = D.weights(lg, 0.005)
    assert dead.tolist() == [True, True, False, False]
    assert w[0] == 0 and w[1] == 0 and w[2] == 1 << 23
    assert abs(w[3] / (1 << 24) - 1 / (1 + math.exp(-4.0))) < 1e-6


# ---------------------------------------------------------------- adaptive density control
def _stats(N):
    return np.zeros(N, np.float32), np.zeros(N, np.float32), np.zeros(N, np.float32)


def test_adc_branches_by_hand():
    g = _gaussians(6, seed=1)
    g.opacity_logits[:] = 2.0
    g.log_scales[:] = math.log(0.005)
    g.log_scales[0, 2] = math.log(0.02)           # big: its largest axis is above split_scale
    g.opacity_logits[3] = math.log(0.004 / 0.996)  # below min_opacity 0.005
    grad, count, radius = _stats(6)
    count[:] = 4
    grad[:] = 4 * 1e-4                              # mean 1e-4 < threshold
    grad[1] = 4 * 2e-4                              # mean == threshold: dense (>=)
    grad[2] = 4 * 3e-4                              # dense and big: split
    grad[4] = 4 * 5e-4
    count[4] = 0                                    # no views: mean 0, not dense
    radius[5] = 30.0                                # above max_screen_radius 20
    normals = np.zeros((2, 3, 6), np.float32)
    d = D.adc_decisions(g, grad, count, radius, 2e-4, 0.01, 0.005, max_screen_radius=20.0)
    assert d["pruned"].tolist() == [False, False, False, True, False, True]
    assert d["clone"].tolist() == [False, True, False, False, False, False]
    assert d["split"].tolist() == [False, False, True, False, False, False]
    out = D.adc(g, grad, count, radius, normals, 2e-4, 0.01, 0.005, max_screen_radius=20.0)
    # kept 0; 1 and its clone; the two children of 2 (at its mean for zero draws); 4 kept
    assert out.N == 6
    g64 = g.as64()
    for k, src in enumerate([0, 1, 1, 2, 2, 4]):
        np.testing.assert_array_equal(out.means[:, k], g64.means[:, src])
        np.testing.assert_array_equal(out.sh[:, k], g64.sh[:, src])
        np.testing.assert_array_equal(out.opacity_logits[k], g64.opacity_logits[src])
        if src == 2:
            np.testing.assert_allclose(out.log_scales[:, k], g64.log_scales[:, 2] - math.log(1.6), rtol=0,
                                       atol=1e-15)
        else:
            np.testing.assert_array_equal(out.log_scales[:, k], g64.log_scales[:, src])


def test_adc_split_children_sit_at_mean_plus_R_S_eps():
    rng = np.random.default_rng(3)
    g = _gaussians(5, seed=3)
    g.opacity_logits[:] = 3.0
    grad, count, radius = _stats(5)
    count[:] = 1
    grad[:] = 1.0
    normals = rng.normal(0, 1, (2, 3, 5)).astype(np.float32)
    out = D.adc(g, grad, count, radius, normals, 1e-4, 1e-6, 0.005)   # every Gaussian dense and big
    assert out.N == 10
    q = g.quats.astype(np.float64)
    for i in range(5):
        R = Rotation.from_quat([q[1, i], q[2, i], q[3, i], q[0, i]]).as_matrix()   # scipy: (x, y, z, w)
        S = np.diag(np.exp(g.log_scales[:, i].astype(np.float64)))
        for c in range(2):
            want = g.means[:, i].astype(np.float64) + R @ S @ normals[c, :, i].astype(np.float64)
            np.testing.assert_allclose(out.means[:, 2 * i + c], want, rtol=0, atol=1e-12)


def test_adc_world_scale_prune_and_thresholds_compare_exactly():
    g = _gaussians(3, seed=4)
    g.opacity_logits[:] = 1.0
    g.log_scales[:] = -5.0
    g.log_scales[1, 1] = np.float32(math.log(0.5)) + np.float32(1e-6)   # just above max_world_scale 0.5
    grad, count, radius = _stats(3)
    d = D.adc_decisions(g, grad, count, radius, 1e-3, 0.01, 0.005, max_world_scale=0.5)
    assert d["pruned"].tolist() == [False, True, False]
    assert d["n_out"].tolist() == [1, 0, 1]


# ---------------------------------------------------------------- MCMC relocation
@pytest.mark.parametrize("o", [0.01, 0.3, 0.8, 0.99])
@pytest.mark.parametrize("k", [1, 2, 3, 5])
def test_relocated_copies_stack_to_the_original_opacity(o, k):
    on = float(D.relocation_opacity(o, k))
    assert 1 - (1 - on) ** k == pytest.approx(o, rel=1e-12)


@pytest.mark.parametrize("o", [0.05, 0.5, 0.95])
@pytest.mark.parametrize("k", [1, 2, 3, 6])
def test_relocated_scale_keeps_the_integral_of_the_opacity_profile(o, k):
    """k copies of opacity o' and width c sigma, composited, integrate (along a
    line through the centre) to the original o exp(-x^2 / 2 sigma^2)."""
    on = float(D.relocation_opacity(o, k))
    c = D.relocation_scale_factor(o, on, k)
    stacked, _ = integrate.quad(lambda x: 1 - (1 - on * math.exp(-x * x / (2 * c * c))) ** k, -60, 60,
                                limit=200)
    single, _ = integrate.quad(lambda x: o * math.exp(-x * x / 2), -60, 60, limit=200)
    assert stacked == pytest.approx(single, rel=1e-9)
    if k == 1:
        assert c == pytest.approx(1.0, rel=1e-14)


def test_relocation_sources_by_hand():
    # weights: dead, 2^23 (sigma 0.5), dead, 2^23 -> W = 2^24; t = floor(r W / 2^32)
    lg = np.array([-9.0, 0.0, -9.0, 0.0], np.float32)
    r = np.zeros(4, np.uint64)
    r[0] = (1 << 31) - 1        # t just below 2^23: the first live source
    r[2] = 1 << 31              # t = 2^23: the second
    dead, src, drawn = D.relocate_sources(lg, r, 0.005)
    assert dead.tolist() == [True, False, True, False]
    assert src.tolist() == [1, -1, 3, -1]
    assert drawn.tolist() == [0, 1, 0, 1]


def test_relocation_draws_follow_the_opacities():
    rng = np.random.default_rng(7)
    lg = np.full(2000, -9.0, np.float32)             # 1994 dead slots
    live = [10, 500, 1200, 1999, 3, 700]
    o = np.array([0.9, 0.6, 0.3, 0.15, 0.05, 0.02])
    lg[live] = np.log(o / (1 - o)).astype(np.float32)
    r = rng.integers(0, 1 << 32, 2000, dtype=np.uint64)
    _, src, drawn = D.relocate_sources(lg, r, 0.005)
    assert (src[live] == -1).all() and drawn.sum() == 2000 - len(live)
    freq = drawn[live] / drawn.sum()
    np.testing.assert_allclose(freq, o / o.sum(), atol=0.03)


def test_relocate_moves_dead_onto_updated_sources():
    g = _gaussians(6, seed=8)
    g.opacity_logits[:] = np.array([2.0, -9.0, 1.0, -9.0, -9.0, 0.5], np.float32)
    r = np.array([0, 7 << 28, 0, 1 << 20, 15 << 28, 0], np.uint64)
    out, src = D.mcmc_relocate(g, r, 0.005)
    dead = [1, 3, 4]
    for d in dead:
        s = src[d]
        assert s in (0, 2, 5)
        for name in ("means", "quats", "sh"):
            np.testing.assert_array_equal(getattr(out, name)[..., d], getattr(g.as64(), name)[..., s])
        np.testing.assert_array_equal(out.opacity_logits[d], out.opacity_logits[s])
        np.testing.assert_array_equal(out.log_scales[:, d], out.log_scales[:, s])
    for s in (0, 2, 5):
        k = 1 + int((src == s).sum())
        o = D.sigmoid(g.opacity_logits[s])
        assert 1 - (1 - D.sigmoid(out.opacity_logits[s])) ** k == pytest.approx(o, rel=1e-9)


def test_relocate_without_live_gaussians_changes_nothing():
    g = _gaussians(4, seed=9)
    g.opacity_logits[:] = -9.0
    out, src = D.mcmc_relocate(g, np.arange(4, dtype=np.uint64) << 30, 0.005)
    assert (src == -1).all()
    np.testing.assert_array_equal(out.means, g.as64().means)
    np.testing.assert_array_equal(out.opacity_logits, g.as64().opacity_logits)


# ---------------------------------------------------------------- MCMC noise
def test_noise_step_is_gated_covariance_times_draw():
    g = _gaussians(3, seed=10)
    g.opacity_logits[:] = np.array([math.log(0.005 / 0.995), 8.0, -1.0], np.float32)
    for axis in range(3):
        eta = np.zeros((3, 3))
        eta[axis] = 1.0
        new = D.mcmc_noise(g, eta, 2.0)
        step = new - g.as64().means
        q = g.quats.astype(np.float64)
        for i in range(3):
            R = Rotation.from_quat([q[1, i], q[2, i], q[3, i], q[0, i]]).as_matrix()
            Sigma = R @ np.diag(np.exp(2 * g.log_scales[:, i].astype(np.float64))) @ R.T
            o = 1 / (1 + math.exp(-float(g.opacity_logits[i])))
            gate = 1 / (1 + math.exp(100 * (o - 0.005)))
            np.testing.assert_allclose(step[:, i], 2.0 * gate * Sigma[:, axis], rtol=1e-9, atol=1e-15)
    # at the threshold opacity the gate is one half; an opaque Gaussian barely moves
    o0 = 1 / (1 + math.exp(-float(g.opacity_logits[0])))
    assert 1 / (1 + math.exp(100 * (o0 - 0.005))) == pytest.approx(0.5, abs=1e-6)
