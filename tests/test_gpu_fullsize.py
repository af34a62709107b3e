"""Full-size parity on the benchmark workload (8 keyframes x 640x480 into 8 views) in
the launch configuration bench.py times: the library's autotuner picks the work split on
this scene, as the benchmark does before timing (persistent heavy-first schedules, the
batches it chooses); the split the benchmark reported (16x16 tiles, batches 512 / 512,
both passes persistent) is run too. The oracle cannot render all of it in test time, so
it checks sampled tile lists entry by entry, sampled pixels and sampled Gaussians one by
one, the exact key count, and properties that hold at any size; every split must render
what the default split of its tile shape renders, bit for bit."""
import numpy as np
import pytest

import oracle
from parity import gpu_run

pytestmark = pytest.mark.gpu

BENCH_SPLIT = dict(fwd_batch=512, bwd_batch=512, fwd_schedule="persistent", bwd_schedule="persistent")


def _tuned_options(scene, grads):
    import torch
    from paper_2603_21055_gb300 import splat
    sp = splat.Splatter()
    kfs = splat.upload_keyframes(scene)
    sp.plan(kfs, scene.views)
    images = splat.alloc_images(scene.views)
    gin = [{k: torch.as_tensor(v).cuda() for k, v in g.items()} for g in grads]
    gout = [dict(d_offset=torch.empty_like(k.offset), d_rgb=torch.empty_like(k.rgb), d_logit=torch.empty_like(k.logit),
                 d_scale=torch.empty_like(k.scale)) for k in kfs]
    sp.autotune(kfs, scene.views, images, gin, gout, reps=3)
    return sp.options


@pytest.fixture(scope="module")
def full(room2):
    rng = np.random.default_rng(11)
    # image gradients: the L1 gradient of the paper's loss against the observations needs
    # the rendered images; use fixed seeded gradients of the same magnitude instead
    grads = []
    for v in room2.views:
        hw = v.width * v.height
        grads.append(dict(rgb=(np.sign(rng.normal(size=(3, v.height, v.width))) / (3 * hw)).astype(np.float32),
                          depth=(0.1 * np.sign(rng.normal(size=(v.height, v.width))) / hw).astype(np.float32)))
    opts = _tuned_options(room2, grads)
    res = gpu_run(room2, grads_in=grads, options=opts)
    tile = (opts.tile_w, opts.tile_h)
    print("autotuned split: tile %dx%d, forward batch %d schedule %d, backward algorithm %d batch %d schedule %d" %
          (tile + (opts.fwd_batch, opts.fwd_schedule, opts.bwd_algorithm, opts.bwd_batch, opts.bwd_schedule)))
    return dict(res=res, grads=grads, tile=tile, o=oracle.opts(tile_w=tile[0], tile_h=tile[1]))


def _same_forward(a, b):
    for ia, ib in zip(a["images"], b["images"]):
        for q in ("rgb", "depth", "alpha"):
            np.testing.assert_array_equal(ia[q], ib[q])
    np.testing.assert_array_equal(a["n_contrib"], b["n_contrib"])
    np.testing.assert_array_equal(a["t_final"], b["t_final"])
    np.testing.assert_array_equal(a["entries"], b["entries"])


def _close_grads(a, b):
    for ga, gb in zip(a["grads"], b["grads"]):
        for q in ("d_offset", "d_rgb", "d_logit", "d_scale"):
            x, y = ga[q].astype(np.float64), gb[q].astype(np.float64)
            assert np.all(np.isfinite(x)), q
            assert np.linalg.norm(x - y) <= 1e-5 * np.linalg.norm(y), q
            assert np.abs(x - y).max() <= 1e-4 * np.abs(y).max(), q


def test_splits_match_default(room2, full):
    """The autotuned split and the benchmark's reported split against the default split
    (one block per tile) of the same tile shape."""
    base = gpu_run(room2, grads_in=full["grads"], tile=full["tile"])
    _same_forward(full["res"], base)
    _close_grads(full["res"], base)
    bench = gpu_run(room2, grads_in=full["grads"], **BENCH_SPLIT)
    base16 = base if full["tile"] == (16, 16) else gpu_run(room2, grads_in=full["grads"])
    _same_forward(bench, base16)
    _close_grads(bench, base16)


def test_key_count_exact(room2, full):
    res, o = full["res"], full["o"]
    total, near = 0, 0
    for k in range(len(room2.views)):
        P = oracle.project(room2, k, o)
        total += int(P["ntiles"].sum())
        near += int(P["ntiles"][P["near"] != 0].sum())
    assert abs(res["n_keys"] - total) <= near, (res["n_keys"], total, near)


def test_sampled_tile_lists(room2, full):
    """The sorted lists of 50 full-size tiles (the 10 longest and 40 at random) entry by
    entry against the definition: every Gaussian whose tile rectangle holds the tile,
    ordered by (depth rounded to f32, index). (View, Gaussian) pairs with a near binning
    or key-rounding decision are set aside on both sides."""
    res, o = full["res"], full["o"]
    tw, th = full["tile"]
    offs, ent = res["offsets"], res["entries"]
    lengths = np.diff(offs)
    rng = np.random.default_rng(12)
    longest = np.argsort(lengths)[::-1][:10]
    pick = np.unique(np.concatenate([longest, rng.choice(len(lengths), 40, replace=False)]))
    v0 = room2.views[0]
    per_view = ((v0.width + tw - 1) // tw) * ((v0.height + th - 1) // th)
    tiles_x = (v0.width + tw - 1) // tw
    checked, aside = 0, 0
    for k in np.unique(pick // per_view):
        P = oracle.project(room2, int(k), o)
        zbits = P["zf"].astype(np.float32).view(np.uint32)
        for t in pick[pick // per_view == k]:
            local = int(t) - int(k) * per_view
            tx, ty = local % tiles_x, local // tiles_x
            cov = (P["ntiles"] > 0) & (P["tx0"] <= tx) & (P["tx1"] >= tx) & (P["ty0"] <= ty) & (P["ty1"] >= ty)
            g = np.nonzero(cov)[0]
            order = np.lexsort((g, zbits[g]))
            ref_g, ref_z = g[order], zbits[g][order]
            gl = ent[offs[t]:offs[t + 1]]
            got_g = (gl & np.uint64(0xffffffff)).astype(np.int64)
            got_z = (gl >> np.uint64(32)).astype(np.uint32)
            near = P["near"] != 0
            keep_ref, keep_got = ~near[ref_g], ~near[got_g]
            aside += int((~keep_ref).sum())
            np.testing.assert_array_equal(got_g[keep_got], ref_g[keep_ref], err_msg="tile %d" % t)
            np.testing.assert_array_equal(got_z[keep_got], ref_z[keep_ref], err_msg="tile %d" % t)
            checked += int(keep_ref.sum())
    print("sampled tile lists: %d tiles, %d entries equal, %d set aside; longest %d" %
          (len(pick), checked, aside, int(lengths.max())))
    assert aside <= 0.01 * max(checked, 1)


def test_sampled_pixels(room2, full):
    res, o = full["res"], full["o"]
    rng = np.random.default_rng(5)
    n = 400
    vi = rng.integers(0, len(room2.views), n)
    xs = rng.integers(0, 640, n)
    ys = rng.integers(0, 480, n)
    ref = oracle.render_pixels(room2, vi, xs, ys, o)
    clean = ref["near"] == 0
    assert clean.sum() >= 0.9 * n
    for i in np.nonzero(clean)[0]:
        im = res["images"][vi[i]]
        got = np.array([im["rgb"][c, ys[i], xs[i]] for c in range(3)])
        np.testing.assert_allclose(got, ref["rgb"][i], atol=1e-4)
        assert abs(im["depth"][ys[i], xs[i]] - ref["depth"][i]) <= 1e-4
        assert abs(im["alpha"][ys[i], xs[i]] - ref["alpha"][i]) <= 1e-4
        p = vi[i] * 640 * 480 + ys[i] * 640 + xs[i]
        assert res["n_contrib"][p] == ref["n_contrib"][i]


def test_sampled_gaussian_gradients(room2, full):
    res, grads, o = full["res"], full["grads"], full["o"]
    rng = np.random.default_rng(6)
    sel = rng.choice(room2.n_gaussians, 60, replace=False)
    ref, near, absum = oracle.backward_gaussians(room2, [{k: v.astype(np.float64) for k, v in g.items()}
                                                         for g in grads], sel, o)
    names = ("d_offset", "d_rgb", "d_rgb", "d_rgb", "d_logit", "d_scale")
    scale = np.abs(ref).max(axis=0)
    for s, g in enumerate(sel):
        if near[s]:
            continue
        kf, j = divmod(int(g), 640 * 480)
        y, x = divmod(j, 640)
        gk = res["grads"][kf]
        got = [gk["d_offset"][y, x], gk["d_rgb"][0, y, x], gk["d_rgb"][1, y, x], gk["d_rgb"][2, y, x],
               gk["d_logit"][y, x], gk["d_scale"][y, x]]
        for q in range(6):
            tol = 1e-3 * abs(ref[s, q]) + 1e-4 * absum[s, q] + 1e-6 * scale[q]
            assert abs(got[q] - ref[s, q]) <= tol, (names[q], g, got[q], ref[s, q])


def test_properties_at_full_size(full):
    res = full["res"]
    for im in res["images"]:
        assert np.all(im["alpha"] >= -1e-6) and np.all(im["alpha"] <= 1 + 1e-6)
    t = res["t_final"]
    assert np.all(t >= 1e-4 * (1 - 1e-6)) and np.all(t <= 1.0)
    a = np.concatenate([im["alpha"].ravel() for im in res["images"]])
    np.testing.assert_allclose(a, 1.0 - t, atol=2e-5)
    lengths = np.diff(res["offsets"])
    assert res["n_contrib"].max() <= lengths.max()
