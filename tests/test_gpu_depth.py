"""Depth ray caster (ag_render_depth) against the FP64 oracle.

A pixel whose ray grazes a box silhouette can legitimately be a hit in one
precision and a miss in the other; such pixels are counted and must stay a
small minority (at most 0.01 % of the pixels on the paper-resolution images,
where none was measured; 0.1 % on the 64-box images; 0.2 % on the small
images of the edge cases). Every other pixel must agree to 1e-4 relative.
"""
import math

import numpy as np
import pytest
import torch

import oracle as O
from harness import gpu_fleet
from paper_2305_16510_gb300 import _abi
from paper_2305_16510_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2305_16510_gb300 import build
    build.build()


def _np(t):
    return t.detach().cpu().numpy()


def _compare(gpu, orc, max_bad_frac, check=None, what="pixels beyond 1e-4 relative"):
    close = np.abs(gpu.astype(np.float64) - orc) <= 1e-4 * np.maximum(1.0, orc)
    if check is not None:
        check(what, 1.0 - close.mean(), max_bad_frac)
    assert close.mean() >= 1.0 - max_bad_frac, close.mean()


def test_depth_matches_oracle_small_images():
    w = W.Workload("cams", 300, 1, 0, 16, 300, 0, 0, mode_mix=(0, 1, 2))
    inp = W.make_inputs(w, 12)
    fl = gpu_fleet(w, inp, 12)
    fl.reset(None, 12)
    fl.step(20)
    ids = np.arange(0, 300, 5, dtype=np.int32)
    hfov, rng_max = math.radians(87), 10.0
    img = _np(fl.render_depth(96, 64, hfov, rng_max, cam_offset=(0.1, 0.0, 0.05), env_ids=ids))
    ref = O.render_depth(_np(fl.state()), _np(fl.obstacles()), ids, 96, 64, hfov, rng_max, (0.1, 0.0, 0.05))
    _compare(img, ref, 0.002)
    assert (ref < rng_max).mean() > 0.05          # the cameras really see boxes
    # host destination and default camera ids
    host = np.empty((8, 32, 48), np.float32)
    _abi.ag_render_depth(fl.ctx, 48, 32, hfov, rng_max, None, None, 8, host)
    fl.synchronize()
    ref = O.render_depth(_np(fl.state()), _np(fl.obstacles()), np.arange(8), 48, 32, hfov, rng_max)
    _compare(host, ref, 0.002)
    with pytest.raises(_abi.AgError) as e:
        fl.render_depth(0, 32, hfov, rng_max)
    assert e.value.status == _abi.AG_ERR_INVALID
    with pytest.raises(_abi.AgError):
        _abi.ag_render_depth(fl.ctx, 8, 8, hfov, rng_max, None, np.array([5000], np.uint32), 1, host)
    # a host destination whose staging buffer cannot fit (300 x 2^30 floats, 1.3 TB): AG_ERR_OOM before
    # anything is copied, and the context stays usable
    with pytest.raises(_abi.AgError) as e:
        _abi.ag_render_depth(fl.ctx, 1 << 15, 1 << 15, hfov, rng_max, None, None, 300, host)
    assert e.value.status == _abi.AG_ERR_OOM
    _abi.ag_render_depth(fl.ctx, 48, 32, hfov, rng_max, None, None, 8, host)
    fl.synchronize()
    _compare(host, ref, 0.002)
    # ids out of range in a device array are not read through: those images are NaN, the others unchanged
    dev_ids = torch.tensor([3, 300, 7, -1, 299], dtype=torch.int32, device=fl.device)  # -1: id 2^32 - 1
    img = _np(fl.render_depth(48, 32, hfov, rng_max, env_ids=dev_ids))
    assert np.isnan(img[1]).all() and np.isnan(img[3]).all()
    good = [0, 2, 4]
    ref = O.render_depth(_np(fl.state()), _np(fl.obstacles()), np.array([3, 7, 299]), 48, 32, hfov, rng_max)
    assert not np.isnan(img[good]).any()
    _compare(img[good], ref, 0.002)
    fl.close()


def test_depth_without_boxes_is_max_range_everywhere():
    from paper_2305_16510_gb300.fleet import Fleet
    fl = Fleet(40)
    fl.reset(None, 3)
    img = _np(fl.render_depth(33, 17, math.radians(87), 7.5, cam_offset=(0.1, 0.0, 0.0)))
    assert img.shape == (40, 17, 33)
    assert np.all(img == np.float32(7.5))
    fl.close()


def test_depth_paper_resolution_1024_robots_sampled(within_tolerance):
    # 2^10 robots with 270 x 480 depth cameras (the paper's depth-camera
    # workload); 3 sampled cameras are re-rendered by the oracle
    w = W.Workload("cams", 1024, 4, 1, 16, 1024, 0, 0, mode_mix=(0, 1, 2))
    inp = W.make_inputs(w, 13)
    fl = gpu_fleet(w, inp, 13)
    fl.reset(None, 13)
    fl.step(10)
    img = fl.render_depth(480, 270, math.radians(87), 10.0)
    assert img.shape == (1024, 270, 480)
    assert (img < 10.0).float().mean().item() > 0.05
    st, bx = _np(fl.state()), _np(fl.obstacles())
    for j in (0, 511, 1023):
        ref = O.render_depth(st, bx, [j], 480, 270, math.radians(87), 10.0)
        _compare(_np(img[j:j + 1]), ref, 1e-4, within_tolerance, f"camera {j}: pixels beyond 1e-4 relative")
    fl.close()


def test_depth_with_the_maximum_box_count(within_tolerance):
    # AG_MAX_OBSTACLES boxes per environment, the nearest surface taken over all of them
    n_obs = _abi.AG_MAX_OBSTACLES
    w = W.Workload("cams_many", 4, 1, 0, n_obs, 4, 0, 0)
    inp = W.make_inputs(w, 14)
    fl = gpu_fleet(w, inp, 14)
    fl.reset(None, 14)
    hfov, rng_max = math.radians(70), 20.0
    img = _np(fl.render_depth(40, 24, hfov, rng_max))
    ref = O.render_depth(_np(fl.state()), _np(fl.obstacles()), np.arange(4), 40, 24, hfov, rng_max)
    _compare(img, ref, 1e-3, within_tolerance)
    assert (ref < rng_max).mean() > 0.3
    # the last box alone decides some pixels: moving it away changes them
    boxes = _np(fl.obstacles()).copy()
    boxes[n_obs - 1, 0:3] = 1e6
    fl.set_obstacles(boxes)
    img2 = _np(fl.render_depth(40, 24, hfov, rng_max))
    ref2 = O.render_depth(_np(fl.state()), boxes, np.arange(4), 40, 24, hfov, rng_max)
    _compare(img2, ref2, 0.01)
    fl.close()


def test_depth_more_cameras_than_a_grid_dimension():
    # 70,000 cameras (above the 65,535 limit of a grid's y and z dimensions)
    w = W.Workload("cams_wide", 70000, 1, 0, 2, 70000, 0, 0)
    inp = W.make_inputs(w, 15)
    fl = gpu_fleet(w, inp, 15)
    fl.reset(None, 15)
    hfov, rng_max = math.radians(90), 12.0
    img = _np(fl.render_depth(8, 6, hfov, rng_max))
    ref = O.render_depth(_np(fl.state()), _np(fl.obstacles()), np.arange(w.n_envs), 8, 6, hfov, rng_max)
    _compare(img, ref, 0.002)
    assert (ref[-100:] < rng_max).any()       # the last cameras were rendered too
    fl.close()


def test_depth_full_size_sampled_cameras(within_tolerance):
    """The bench's depth workload (2^10 robots of the obstacle recipe, 16 boxes
    each, after 10 steps, 270 x 480 at 87 deg): 12 sampled cameras are
    rendered again by the oracle, whole."""
    w = W.scaled(W.WORKLOADS["obstacles"], 1024)
    seed = 1
    inp = W.make_inputs(w, seed)
    fl = gpu_fleet(w, inp, seed)
    fl.reset(None, seed)
    fl.step(10)
    hfov, rng_max = math.radians(87), 10.0
    img = fl.render_depth(480, 270, hfov, rng_max)
    state, boxes = _np(fl.state()), _np(fl.obstacles())
    cams = np.sort(np.random.default_rng(3).choice(w.n_envs, 12, replace=False))
    got = _np(img[torch.from_numpy(cams).cuda()])
    fl.close()
    ref = O.render_depth(state, boxes, cams, 480, 270, hfov, rng_max)
    _compare(got, ref, 1e-4, within_tolerance)
    assert (ref < rng_max).mean() > 0.05


def _mismatch(a, b):
    """Fraction of pixels where two float32 images differ by more than 1e-4 relative."""
    a64, b64 = a.astype(np.float64), b.astype(np.float64)
    return float((np.abs(a64 - b64) > 1e-4 * np.maximum(1.0, np.abs(b64))).mean())


def test_fast_reciprocal_moves_few_pixels(within_tolerance):
    """The kernel's fast reciprocals against the same kernel with correctly
    rounded ones (ag_render_depth_ieee), on the bench's depth workload (2^10
    robots, 270 x 480, 16 boxes): 3 of the 132.7 million pixels differ by
    more than 1e-4 relative (2.3e-8), bound 1e-6; against the oracle both
    variants stay within the 1e-4 budget of the full-size comparisons."""
    w = W.scaled(W.WORKLOADS["obstacles"], 1024)
    inp = W.make_inputs(w, 1)
    fl = gpu_fleet(w, inp, 1)
    fl.reset(None, 1)
    fl.step(10)
    hfov, rng_max = math.radians(87), 10.0
    fast = _np(fl.render_depth(480, 270, hfov, rng_max))
    ieee = torch.empty((1024, 270, 480), dtype=torch.float32, device=fl.device)
    _abi.ag_render_depth_ieee(fl.ctx, 480, 270, hfov, rng_max, None, None, 1024, ieee)
    ieee = _np(ieee)
    moved = _mismatch(fast, ieee)
    exact_equal = float((fast == ieee).mean())
    cams = np.sort(np.random.default_rng(4).choice(1024, 8, replace=False))
    ref = O.render_depth(_np(fl.state()), _np(fl.obstacles()), cams, 480, 270, hfov, rng_max)
    fl.close()
    bad_fast, bad_ieee = _mismatch(fast[cams], ref), _mismatch(ieee[cams], ref)
    print(f"fast vs ieee: {100 * moved:.4f} % of pixels beyond 1e-4 rel ({100 * exact_equal:.2f} % bit-equal); "
          f"vs oracle on 8 cameras: fast {100 * bad_fast:.4f} %, ieee {100 * bad_ieee:.4f} %")
    within_tolerance("pixels the fast reciprocal moves beyond 1e-4 relative", moved, 1e-6)
    within_tolerance("fast vs oracle: pixels beyond 1e-4 relative", bad_fast, 1e-4)
    within_tolerance("ieee vs oracle: pixels beyond 1e-4 relative", bad_ieee, 1e-4)
    assert bad_ieee <= bad_fast + 1e-4


def test_live_pair_count_bounds_and_monotone_in_range():
    """ag_depth_live_pairs: at most every (pixel, box) pair, more than none when
    the cameras see boxes, no more at a shorter range, none without boxes, and
    the same on a repeated call."""
    w = W.scaled(W.WORKLOADS["obstacles"], 256)
    inp = W.make_inputs(w, 2)
    fl = gpu_fleet(w, inp, 2)
    fl.reset(None, 2)
    fl.step(5)
    hfov = math.radians(87)
    all_pairs = 256 * 270 * 480 * w.n_obstacles
    live = _abi.ag_depth_live_pairs(fl.ctx, 480, 270, hfov, 10.0, None, None, 256)
    assert 0 < live < all_pairs
    assert _abi.ag_depth_live_pairs(fl.ctx, 480, 270, hfov, 10.0, None, None, 256) == live
    short = _abi.ag_depth_live_pairs(fl.ctx, 480, 270, hfov, 0.5, None, None, 256)
    assert short <= live
    # a live pair is needed for every pixel that sees a box
    img = _np(fl.render_depth(480, 270, hfov, 10.0))
    assert live >= int((img < 10.0).sum())
    fl.close()
    from paper_2305_16510_gb300.fleet import Fleet
    empty = Fleet(16)
    empty.reset(None, 3)
    assert _abi.ag_depth_live_pairs(empty.ctx, 64, 48, hfov, 10.0, None, None, 16) == 0
    empty.close()
