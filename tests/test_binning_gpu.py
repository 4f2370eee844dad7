"""GPU tests of the two tile-binning strategies (include/gsr.h, GSR_BIN_TILE and
GSR_BIN_RADIX): both must give the list order of the oracle -- by tile, then
depth, then Gaussian index -- so their images are bit-identical to each other,
and the per-tile strategy must meet the oracle on scenes whose tiles take each
of its sort paths (a warp's registers, a block's shared memory, the merge of
shared-memory runs) and whose Gaussians tie in depth."""
import dataclasses

import numpy as np
import pytest
import torch

import oracle
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


def _forward(sc, binning, tile=16):
    return U.gpu_forward(sc, rast=R.GaussianRasterizer(tile, binning=binning))


def _assert_same_images(a, b):
    for va, vb in zip(a, b):
        for k in ("color", "depth", "alpha"):
            np.testing.assert_array_equal(va[k], vb[k])


def _clump(N, H=48, W=64, f=60.0, logit=-3.0, log_scale=-1.2, seed=21, pair_ties=True):
    """N Gaussians (SH degree 0) in front of one small view.  With pair_ties,
    Gaussian 2k+1 shares the mean of 2k (equal depth, so only the index
    orders them) but not its shape, opacity or colour."""
    rng = np.random.default_rng(seed)
    z = rng.uniform(2.0, 6.0, N)
    xy = rng.uniform(-0.25, 0.25, (2, N)) * z
    means = np.stack([xy[0], xy[1], z]).astype(np.float32)
    if pair_ties:
        means[:, 1::2] = means[:, 0:N - N % 2:2]
    base = scenes.config_small(seed=seed, N=2, H=H, W=W, f=f)
    return dataclasses.replace(
        base, means=np.ascontiguousarray(means),
        log_scales=np.ascontiguousarray(rng.normal(log_scale, 0.1, (3, N)).astype(np.float32)),
        quats=scenes.random_quats(rng, N),
        opacity_logits=np.ascontiguousarray(rng.normal(logit, 0.2, N).astype(np.float32)),
        sh=scenes.sh_coeffs(rng, N, 0))


@pytest.mark.parametrize("name", list(REDUCED))
def test_strategies_give_identical_images(name):
    sc = REDUCED[name]()
    a, sa = _forward(sc, "tile")
    b, sb = _forward(sc, "radix")
    _assert_same_images(a, b)
    gC, gD, gA = U.upstream(sc)
    ga = U.gpu_backward(sc, sa, gC, gD, gA)
    gb = U.gpu_backward(sc, sb, gC, gD, gA)
    for k in ga:   # the blend's float atomics add in a timing-dependent order
        assert U.rel_l2(ga[k], gb[k]) < 1e-5, k


@pytest.mark.parametrize("name", list(REDUCED))
def test_keys_reserved_in_the_preprocess_match_the_scan(name):
    """Per-tile binning reserves each warp's keys with an atomic, so the
    unsorted keys land in a timing-dependent order: the key count must equal
    the radix path's scan total, and repeated renders must agree bit for bit."""
    sc = REDUCED[name]()
    params, cams, vm = U.to_device(sc)
    counts, images, visible = [], [], []
    for binning in ("radix", "tile", "tile", "tile"):
        rast = R.GaussianRasterizer(16, binning=binning)
        c, d, a, ws = rast.render_forward(params, sc.sh_degree, cams, vm)
        info = rast.info(ws)
        assert info.status == B.OK
        counts.append(info.keys)
        visible.append(info.pairs_visible)
        images.append([t.cpu().numpy() for t in (c, d, a)])
    assert len(set(counts)) == 1 and counts[0] > 0
    # the visible-pair count is the binning's too, and adds up over the views rendered alone
    assert len(set(visible)) == 1 and 0 < visible[0] <= sc.V * sc.N
    alone = 0
    for v in range(sc.V):
        rast = R.GaussianRasterizer(16)
        _, _, _, ws = rast.render_forward(params, sc.sh_degree, cams[v:v + 1], vm[v:v + 1].contiguous())
        alone += rast.info(ws).pairs_visible
    assert alone == visible[0]
    for im in images[2:]:
        for x, y in zip(images[1], im):
            np.testing.assert_array_equal(x, y)


@pytest.mark.parametrize("tile", [8, 16, 32])
def test_strategies_agree_on_every_tile_size(tile):
    sc = REDUCED["uneven"]()
    _assert_same_images(_forward(sc, "tile", tile)[0], _forward(sc, "radix", tile)[0])


def test_block_sort_path_and_depth_ties_against_oracle():
    # 1,500 Gaussians over 12 tiles: most tiles hold more keys than a warp sorts
    sc = _clump(1500)
    got, state = _forward(sc, "tile")
    info = state[0].info(state[4])
    assert info.keys > 12 * 256
    ref = oracle.render(sc)
    flips, n, _ = U.compare_images(ref[0], got[0], "clump")
    assert flips <= max(2, U.FLIP_SHARE * n)
    _assert_same_images(got, _forward(sc, "radix")[0])
    gC, gD, gA = U.upstream(sc)
    g = U.gpu_backward(sc, state, gC, gD, gA)
    _, gref = oracle.render_backward(sc, gC, gD, gA)
    U.compare_grads(gref, g, label="clump")


@pytest.mark.parametrize("N,log_scale", [(1500, -1.2), (8000, -0.6)])
def test_depth_ties_between_distant_ids(N, log_scale):
    """Gaussians k and k + N/2 share their mean (so their depth) but not their
    shape, opacity or colour: far apart in id, they are emitted by different
    warps in either order, and the block and big-tile sorts must still put
    the lower id first (the radix strategy orders them by pair order)."""
    sc = _clump(N, log_scale=log_scale, pair_ties=False)
    h = N // 2
    sc.means[:, h:2 * h] = sc.means[:, :h]
    a, sa = _forward(sc, "tile")
    big = log_scale > -1.0
    assert sa[0].info(sa[4]).keys > 12 * (2048 if big else 256)
    _assert_same_images(a, _forward(sc, "radix")[0])


def test_long_runs_of_equal_depth():
    """40 Gaussians share each of 75 means (ids k, k + 75, ...): runs of 40
    equal depths, too long for the transposition rounds, take the block sort's
    full re-sort from the id digits, and must match the radix strategy."""
    N = 3000
    sc = _clump(N, pair_ties=False)
    sc.means[:] = sc.means[:, np.arange(N) % 75]
    a, sa = _forward(sc, "tile")
    assert sa[0].info(sa[4]).keys > 12 * 256
    _assert_same_images(a, _forward(sc, "radix")[0])


def test_onesweep_tile_grouping_beyond_the_bucket_limit():
    """More than 65,536 tiles (4 views of 1280x1024 at tile 8: 81,920): the
    per-tile strategy groups the keys with the onesweep passes over the tile
    bits instead of the bucket scatter, and must still match the radix one."""
    sc = scenes.config_window(N=3000, V=4, H=1024, W=1280, f=900.0)
    a, sa = _forward(sc, "tile", tile=8)
    assert sa[0].info(sa[4]).tiles > 65536
    _assert_same_images(a, _forward(sc, "radix", tile=8)[0])


def test_merge_sort_path_matches_radix():
    # 40,000 faint Gaussians (sigma ~ 0.011, so that 255 sigma > 1 still
    # leaves a cutoff ellipse) wider than the view: each of the 12 tiles holds
    # 40,000 keys, sorted as shared-memory runs of 16,384 and merged (an odd
    # run included)
    sc = _clump(40000, logit=-4.5, log_scale=1.2)
    a, sa = _forward(sc, "tile")
    assert sa[0].info(sa[4]).keys >= 12 * 32768
    b, _ = _forward(sc, "radix")
    _assert_same_images(a, b)


def test_empty_and_single_key_tiles():
    # one small Gaussian: a single tile holds one key, every other tile none
    sc = _clump(1, log_scale=-5.0, logit=2.0, f=150.0, H=120, W=160)
    sc.means = np.ascontiguousarray(np.array([[0.05], [0.02], [3.0]], np.float32))
    a, sa = _forward(sc, "tile")
    assert sa[0].info(sa[4]).keys == 1
    ref = oracle.render(sc)
    flips, n, _ = U.compare_images(ref[0], a[0], "single")
    assert flips <= 2
    _assert_same_images(a, _forward(sc, "radix")[0])


def test_radix_binning_capacity_overflow_is_reported():
    sc = REDUCED["uneven"]()
    params, cams, vm = U.to_device(sc)
    rast = R.GaussianRasterizer(16, binning="radix")
    small = rast.alloc_workspace(sc.N, cams, key_capacity=3072)
    P = sum(c.H * c.W for c in cams)
    color = torch.empty(3 * P, device="cuda")
    rast.forward_raw(params, sc.sh_degree, cams, vm, small, color, None, None)
    info = rast.info(small)
    assert info.status == B.ECAPACITY and info.keys > info.key_capacity


@pytest.mark.parametrize("tile,binning", [(16, "tile"), (8, "radix"), (16, "radix")])
def test_entry_batch_64_gives_identical_images_and_gradients(tile, binning):
    """The blends staging 64 list entries per warp and round (gsr_config.batch)
    render bit-identical images; the backward's gradients differ only in the
    order of their FP32 sums."""
    for name in ("window", "uneven"):
        sc = REDUCED[name]()
        a, sa = U.gpu_forward(sc, rast=R.GaussianRasterizer(tile, binning=binning, batch=32))
        b, sb = U.gpu_forward(sc, rast=R.GaussianRasterizer(tile, binning=binning, batch=64))
        _assert_same_images(a, b)
        gC, gD, gA = U.upstream(sc)
        ga = U.gpu_backward(sc, sa, gC, gD, gA)
        gb = U.gpu_backward(sc, sb, gC, gD, gA)
        for k in ("means", "log_scales", "quats", "opacity_logits", "sh", "pose"):
            assert U.rel_l2(gb[k], ga[k]) < 1e-5, (name, k)


def test_entry_batch_64_is_refused_at_tile_32():
    with pytest.raises(B.GsrError):
        R.GaussianRasterizer(32, batch=64)


def test_bucket_binning_capacity_overflow_with_tile_order():
    """The default per-tile binning (bucket grouping, blends in most-keys-first
    tile order) on a workspace too small for the keys: only the keys that fit
    are grouped and the ranges are clamped, so the forward and the backward
    stay in bounds and report GSR_ECAPACITY; the same context then renders
    correctly on a workspace with room."""
    sc = REDUCED["uneven"]()
    params, cams, vm = U.to_device(sc)
    rast = R.GaussianRasterizer(16)
    small = rast.alloc_workspace(sc.N, cams, key_capacity=3072)
    P = sum(c.H * c.W for c in cams)
    color, depth, alpha = (torch.empty(3 * P, device="cuda"), torch.empty(P, device="cuda"),
                           torch.empty(P, device="cuda"))
    rast.forward_raw(params, sc.sh_degree, cams, vm, small, color, depth, alpha)
    info = rast.info(small)
    assert info.tiles <= 32768, "the bucket grouping runs up to 32,768 tiles"
    assert info.status == B.ECAPACITY and info.keys > info.key_capacity
    grads = {k: torch.empty_like(v) for k, v in params.items()}
    d_pose = torch.empty(len(cams), 6, device="cuda")
    rast.backward_raw(params, sc.sh_degree, cams, vm, small, torch.ones(3 * P, device="cuda"), None, None,
                      grads, d_pose)
    torch.cuda.synchronize()
    assert rast.info(small).status == B.ECAPACITY
    c2, _, _, ws = rast.render_forward(params, sc.sh_degree, cams, vm)
    assert rast.info(ws).status == B.OK
    ref = U.gpu_forward(sc)[0]
    for v, c in enumerate(R.split_views(c2, cams, 3)):
        np.testing.assert_array_equal(c.cpu().numpy(), ref[v]["color"])


@pytest.mark.parametrize("name", ["window", "uneven"])
def test_strategies_agree_on_surfels(name):
    from tests.test_surfel_gpu import gpu_surfels, surfel_scene
    sc = surfel_scene(name)
    a, _ = gpu_surfels(sc, binning="tile")
    b, _ = gpu_surfels(sc, binning="radix")
    for va, vb in zip(a, b):
        for k in va:
            np.testing.assert_array_equal(va[k], vb[k])
