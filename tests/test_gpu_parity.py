"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the same
seeded float32 inputs.

Bars: sort keys, tile lists and contributor counts bit-exact; images within
1e-4 absolute; gradients within 1e-3 relative (floor 1e-6 x max|grad|). Items whose FP64
decision lies within 1e-5 relative of its threshold may legitimately go either way in
FP32; they are set aside and counted (see oracle/sgad_oracle.h).
"""
import numpy as np
import pytest

import oracle
from parity import (compare_grads, compare_images, compare_keys, compare_pose, gpu_run, grad_stats_line,
                    l1_grads)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def crop(room2):
    """3 keyframes x 100x70 px of the room into 2 views of 120x90 px: several tiles per
    view with ragged right and bottom edges."""
    from paper_2603_21055_gb300.synth import crop_scene
    return crop_scene(room2, (260, 200, 100, 70), (250, 190, 120, 90), n_keyframes=3, n_views=2)


def _grads_for(scene):
    ref = oracle.render(scene)
    loss, g = l1_grads(scene, ref)
    return ref, g


def test_config1_forward_keys_images(scene1):
    ref = oracle.render(scene1)
    res = gpu_run(scene1)
    n_aside = compare_keys(res, scene1)
    worst, n_near = compare_images(res, ref)
    print("config1: keys %d (aside %d), max image err %.2e, near pixels %d" % (res["n_keys"], n_aside, worst, n_near))
    assert res["n_keys"] == res["planned"]


def test_config1_backward(scene1):
    ref, g = _grads_for(scene1)
    res = gpu_run(scene1, grads_in=g)
    og = oracle.backward(scene1, [{k: v.astype(np.float64) for k, v in x.items()} for x in g])
    e = compare_grads(res, og)
    print("config1 grad error ratio %.3f" % e)
    print(grad_stats_line("config1"))
    assert e <= 1.0


def test_crop_forward_backward(crop):
    ref, g = _grads_for(crop)
    res = gpu_run(crop, grads_in=g)
    assert res["n_sort_exact"] == 0           # every tile through the one-pass bucket sort
    n_aside = compare_keys(res, crop)
    worst, n_near = compare_images(res, ref)
    og = oracle.backward(crop, [{k: v.astype(np.float64) for k, v in x.items()} for x in g])
    e = compare_grads(res, og)
    print("crop: keys %d aside %d img %.2e near px %d grad ratio %.3f" % (res["n_keys"], n_aside, worst, n_near, e))
    print(grad_stats_line("crop"))
    assert e <= 1.0


@pytest.mark.parametrize("algo", ["pairs", "warp_reduce", "warp_local"])
def test_backward_algorithms(scene1, crop, algo):
    """Every backward algorithm against the oracle, on the plane and the room crop, and
    under the persistent schedule with a grid of 3 blocks (each block, or each of its
    warps, takes many tiles from the queue)."""
    for sc in (scene1, crop):
        ref, g = _grads_for(sc)
        og = oracle.backward(sc, [{k: v.astype(np.float64) for k, v in x.items()} for x in g])
        for split in (dict(), dict(bwd_schedule="persistent", fwd_schedule="persistent", max_blocks=3)):
            res = gpu_run(sc, grads_in=g, bwd_algorithm=algo, **split)
            e = compare_grads(res, og)
            print(grad_stats_line("%s %s %s" % (sc.name, algo, "capped persistent" if split else "tiles")))
            assert e <= 1.0


@pytest.mark.parametrize("tile", [(8, 32), (32, 8)])
def test_crop_other_tile_shapes(crop, tile):
    o = oracle.opts(tile_w=tile[0], tile_h=tile[1])
    ref = oracle.render(crop, o)
    loss, g = l1_grads(crop, ref)
    res = gpu_run(crop, grads_in=g, tile=tile)
    compare_keys(res, crop, o)
    compare_images(res, ref)
    og = oracle.backward(crop, [{k: v.astype(np.float64) for k, v in x.items()} for x in g], o)
    assert compare_grads(res, og) <= 1.0


def test_global_memory_sort_path(crop):
    """Buckets larger than the shared-memory capacity are sorted in chunks and merged
    through global memory; force that path with a 64-entry capacity."""
    ref = oracle.render(crop)
    res = gpu_run(crop, sort_smem_cap=64)
    assert np.diff(res["offsets"]).max() > 64 * 4
    compare_keys(res, crop)
    compare_images(res, ref)


@pytest.mark.parametrize("cap", [100, 6145, 12288])
def test_sort_capacities(crop, cap):
    """Shared-memory sort capacities other than the default 6144: a small one (chunks of
    100 merged through global memory) and the larger ones served by 24 entries per
    thread."""
    res = gpu_run(crop, sort_smem_cap=cap)
    compare_keys(res, crop)


def test_background_and_zero_opacity(scene1):
    """All opacities at zero: the image is exactly the background, nothing contributes,
    every gradient but colour-free terms is zero."""
    from paper_2603_21055_gb300.synth import Keyframe, Scene
    k = scene1.keyframes[0]
    dead = Keyframe(k.cam, k.depth, k.offset, k.rgb, np.full_like(k.logit, -60.0), k.scale)
    sc = Scene([dead], scene1.views, scene1.target_rgb, scene1.target_depth)
    g = [dict(rgb=np.ones((3, 48, 64), np.float32), depth=np.ones((48, 64), np.float32),
              alpha=np.ones((48, 64), np.float32))]
    res = gpu_run(sc, grads_in=g, bg=(0.25, 0.5, 0.75))
    im = res["images"][0]
    for c, b in enumerate((0.25, 0.5, 0.75)):
        assert np.all(im["rgb"][c] == np.float32(b))
    assert np.all(im["alpha"] == 0) and np.all(im["depth"] == 0)
    assert np.all(res["n_contrib"] == 0) and np.all(res["t_final"] == 1)
    for q in ("d_offset", "d_rgb", "d_scale"):
        assert np.all(res["grads"][0][q] == 0)


@pytest.mark.parametrize("algo", ["pairs", "warp_reduce", "warp_local"])
def test_background_and_alpha_gradient(crop, algo):
    """The general compositing adjoint, where Gaussians contribute: a grey background
    (the T_final * background term of every colour channel) and a gradient on the alpha
    image (the alpha suffix sums), against the oracle rendering with the same background;
    for the warp-local backward also the alpha gradient alone on a black background. Both
    under the default schedule and the capped persistent one."""
    rng = np.random.default_rng(17)
    cases = [(0.25, 0.5, 0.75)] + ([(0.0, 0.0, 0.0)] if algo == "warp_local" else [])
    for bg in cases:
        o = oracle.opts(bg=bg)
        ref = oracle.render(crop, o)
        _, g = l1_grads(crop, ref)
        for x, v in zip(g, crop.views):
            x["alpha"] = (rng.choice([-1.0, 1.0], size=(v.height, v.width)) / (v.width * v.height)).astype(np.float32)
        og = oracle.backward(crop, [{k: v.astype(np.float64) for k, v in x.items()} for x in g], o)
        for split in (dict(), dict(bwd_schedule="persistent", fwd_schedule="persistent", max_blocks=3)):
            res = gpu_run(crop, grads_in=g, bg=bg, bwd_algorithm=algo, **split)
            worst, n_near = compare_images(res, ref)
            e = compare_grads(res, og)
            print("bg %s %s %s: img %.2e near px %d grad ratio %.3f"
                  % (bg, algo, "capped persistent" if split else "tiles", worst, n_near, e))
            print(grad_stats_line("bg %s %s" % (bg, algo)))
            assert e <= 1.0


def test_fixed_keyframe_and_frozen_offset(crop):
    """Sec. 3.2: neighbour keyframes are fixed; Table 9 Mode3 freezes delta. A fixed
    keyframe renders identically and gets no gradient; freezing delta zeroes only
    d_offset."""
    from paper_2603_21055_gb300.synth import Keyframe, Scene
    kfs = list(crop.keyframes)
    k1 = kfs[1]
    kfs[1] = Keyframe(k1.cam, k1.depth, k1.offset, k1.rgb, k1.logit, k1.scale, learnable=False)
    sc = Scene(kfs, crop.views, crop.target_rgb, crop.target_depth, crop.depth_weight)
    ref, g = _grads_for(sc)
    a = gpu_run(sc, grads_in=g)
    b = gpu_run(sc, grads_in=g, freeze_offset=True)
    assert a["grads"][1] is None
    np.testing.assert_array_equal(a["images"][0]["rgb"], b["images"][0]["rgb"])
    assert np.all(b["grads"][0]["d_offset"] == 0)
    og = oracle.backward(sc, [{k: v.astype(np.float64) for k, v in x.items()} for x in g])
    assert compare_grads(a, og) <= 1.0
    for q in ("d_rgb", "d_logit", "d_scale"):
        np.testing.assert_allclose(b["grads"][0][q], a["grads"][0][q], rtol=1e-4, atol=1e-7)


def test_key_overflow_is_reported_not_faulted(scene1):
    """A workspace with too few key slots: the forward leaves the outputs untouched and
    sgad_check reports SGAD_ERR_KEY_OVERFLOW with the count needed; a re-plan succeeds."""
    import torch
    from paper_2603_21055_gb300 import binding as B
    from paper_2603_21055_gb300 import splat
    sp = splat.Splatter()
    kfs = splat.upload_keyframes(scene1)
    n = sp.plan(kfs, scene1.views)
    sp.reserve(kfs, scene1.views, n // 2)
    sp.key_capacity = n // 2
    images = splat.alloc_images(scene1.views)
    for im in images:
        for t in im.values():
            t.fill_(-7.0)
    sp.forward(kfs, scene1.views, images)
    status, nk, need = sp.check()
    assert status == B.SGAD_ERR_KEY_OVERFLOW and need == n
    assert torch.all(images[0]["rgb"] == -7.0)
    sp.reserve(kfs, scene1.views, need)
    sp.forward(kfs, scene1.views, images)
    assert sp.check()[0] == 0


def test_invalid_arguments_return_status(scene1):
    from paper_2603_21055_gb300 import binding as B
    from paper_2603_21055_gb300 import splat
    sp = splat.Splatter()
    kfs = splat.upload_keyframes(scene1)
    sp.plan(kfs, scene1.views)
    ka, va = sp.kf_structs(kfs), sp.view_structs(scene1.views)
    out = (B.sgad_images * 1)()
    lib = B.load()
    assert lib.sgad_forward(sp.ctx, ka, 1, va, 0, out, sp.ws_ptr, sp.ws_bytes, sp.key_capacity, None) == \
        B.SGAD_ERR_INVALID_ARG
    assert lib.sgad_forward(sp.ctx, ka, 1, va, 1, out, sp.ws_ptr, 1024, sp.key_capacity, None) == \
        B.SGAD_ERR_WORKSPACE_TOO_SMALL
    assert lib.sgad_forward(sp.ctx, ka, 1, va, 1, out, sp.ws_ptr, sp.ws_bytes, sp.key_capacity, None) == \
        B.SGAD_ERR_INVALID_ARG            # NULL output images


@pytest.mark.parametrize("algo", ["warp_reduce", "pairs", "warp_local"])
def test_view_pose_gradient(scene1, crop, algo):
    """d loss / d (world->cam 3x4) of every view against the oracle's pose adjoint, on the
    plane and on the two-view room crop, with both backward algorithms."""
    for sc in (scene1, crop):
        ref, g = _grads_for(sc)
        res = gpu_run(sc, grads_in=g, pose=True, bwd_algorithm=algo)
        dp, ab = oracle.backward_pose(sc, [{k: v.astype(np.float64) for k, v in x.items()} for x in g])
        e = compare_pose(res, dp, ab)
        print("%s %s pose grad ratio %.3f" % (sc.name, algo, e))
        assert e <= 1.0


def test_view_that_sees_nothing(scene1):
    """A view turned away from every Gaussian: no keys, background images, and every
    gradient written as zero (the outputs start as NaN)."""
    from paper_2603_21055_gb300.synth import Camera, Scene, _f32pose
    v = scene1.views[0]
    P = np.asarray(v.pose, np.float64)
    flip = np.diag([-1.0, 1.0, -1.0])                      # 180 degrees about the camera's y axis
    away = Camera(v.width, v.height, v.fx, v.fy, v.cx, v.cy, _f32pose(np.hstack([flip @ P[:, :3], (flip @ P[:, 3])[:, None]])))
    sc = Scene(scene1.keyframes, [away], scene1.target_rgb, scene1.target_depth, 0.0)
    ref, g = _grads_for(sc)
    res = gpu_run(sc, grads_in=g)
    assert res["n_keys"] == 0
    im = res["images"][0]
    assert not im["rgb"].any() and not im["depth"].any() and not im["alpha"].any()
    assert not np.abs(ref[0]["rgb"]).any()
    for gk in res["grads"]:
        for name, arr in gk.items():
            assert np.isfinite(arr).all() and not arr.any(), name


def test_most_keyframes_and_views(scene1):
    """The most keyframes (32) and views (64) a call takes: disjoint 8 x 6 crops of the
    plane's keyframe and view, so most views see a handful of Gaussians and some none."""
    from paper_2603_21055_gb300.synth import Scene, crop_scene
    kfs, views, tr, td = [], [], [], []
    for i in range(32):
        c = crop_scene(scene1, (8 * (i % 8), 6 * (i // 8), 8, 6), (0, 0, 8, 6))
        kfs += c.keyframes
    for j in range(64):
        c = crop_scene(scene1, (0, 0, 8, 6), (8 * (j % 8), 6 * (j // 8), 8, 6))
        views += c.views
        tr += c.target_rgb
        td += c.target_depth
    sc = Scene(kfs, views, tr, td, 0.0)
    ref, g = _grads_for(sc)
    res = gpu_run(sc, grads_in=g)
    n_aside = compare_keys(res, sc)
    worst, n_near = compare_images(res, ref)
    og = oracle.backward(sc, [{k: v.astype(np.float64) for k, v in x.items()} for x in g])
    e = compare_grads(res, og)
    print("32 kf x 64 views: keys %d aside %d img %.2e grad ratio %.3f" % (res["n_keys"], n_aside, worst, e))
    print(grad_stats_line("32kf x 64 views"))
    assert res["n_keys"] > 0 and e <= 1.0


@pytest.mark.parametrize("quantum", [0.0, 0.001, 0.05])
def test_equal_depth_runs(scene1, quantum):
    """Entries of equal depth in one tile are listed by index. The plane's keyframe is
    seen from its own camera with zero offsets, so an entry's depth is its depth-map
    value: a constant map (every entry of a tile at one depth, long runs) and the tilted
    plane's depths rounded to 1 mm (short runs of equal depth) and to 5 cm (long runs)."""
    from paper_2603_21055_gb300.synth import Camera, Keyframe, Scene
    k = scene1.keyframes[0]
    if quantum == 0.0:
        depth = np.full_like(k.depth, 1.5)
    else:
        depth = (np.round(k.depth / quantum) * quantum).astype(np.float32)
    kf = Keyframe(k.cam, depth, np.zeros_like(k.offset), k.rgb, k.logit, (depth / np.float32(k.cam.fx)).astype(np.float32))
    c = k.cam
    view = Camera(c.width, c.height, c.fx, c.fy, c.cx, c.cy, np.eye(4, dtype=np.float32)[:3].copy())
    sc = Scene([kf], [view], scene1.target_rgb, scene1.target_depth, 0.0)
    ref = oracle.render(sc)
    res = gpu_run(sc)
    offs, ent = res["offsets"], res["entries"]
    runs = 0
    for t in range(len(offs) - 1):
        z = ent[offs[t]:offs[t + 1]] >> np.uint64(32)
        runs = max(runs, int(np.unique(z, return_counts=True)[1].max()) if len(z) else 0)
    assert runs > (32 if quantum != 0.001 else 1)                      # the case it is meant to exercise
    compare_keys(res, sc)
    compare_images(res, ref)
    if quantum == 0.0:
        assert res["n_sort_exact"] > 0        # buckets of equal depths: the exact radix sort
