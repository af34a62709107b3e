"""Helpers shared by the GPU parity tests: run the CUDA path through the C ABI and the
FP64 oracle on the same float32 inputs, and compare them."""
from __future__ import annotations

import numpy as np

import oracle

IMAGE_ATOL = 1e-4          # tolerance for rendered images (absolute)
GRAD_RTOL = 1e-3           # tolerance for gradients (relative)


def gpu_run(scene, grads_in=None, tile=(16, 16), sort_smem_cap=0, freeze_offset=False, bg=(0.0, 0.0, 0.0),
            pose=False, **work_split):
    """Forward (and backward when grads_in is given) through libsgad. Returns a dict of
    numpy results plus the raw forward state. pose: also request each view's pose
    gradient (res["pose"], (n_views, 3, 4)). work_split: fwd_batch, bwd_batch,
    fwd_schedule, bwd_schedule, bwd_algorithm, max_blocks of the Splatter, or options=
    a complete sgad_options (e.g. a tuned one)."""
    import torch
    from paper_2603_21055_gb300 import splat
    sp = splat.Splatter(tile=tile, sort_smem_cap=sort_smem_cap, freeze_offset=freeze_offset, bg=bg, **work_split)
    kfs = splat.upload_keyframes(scene)
    n_keys = sp.plan(kfs, scene.views)
    images = splat.alloc_images(scene.views)
    sp.forward(kfs, scene.views, images)
    status, nk, need = sp.check()
    assert status == 0, (status, nk, need)
    offs, entries, t_final, n_contrib = sp.state(kfs, scene.views)
    stats = sp.stats()
    res = dict(images=[{k: v.cpu().numpy() for k, v in im.items()} for im in images], n_sort_exact=stats["n_sort_exact"],
               offsets=offs.cpu().numpy().astype(np.int64) & 0xffffffff,
               entries=entries.cpu().numpy().view(np.uint64), t_final=t_final.cpu().numpy(),
               n_contrib=n_contrib.cpu().numpy(), n_keys=nk, planned=n_keys)
    if grads_in is not None:
        gin = [{k: torch.as_tensor(np.ascontiguousarray(v, np.float32)).cuda() for k, v in g.items()}
               for g in grads_in]
        if pose:
            for g in gin:
                g["pose"] = torch.full((12,), float("nan"), device="cuda")
        gout = []
        for k in kfs:
            if k.learnable:
                gout.append(dict(d_offset=torch.full_like(k.offset, np.nan), d_rgb=torch.full_like(k.rgb, np.nan),
                                 d_logit=torch.full_like(k.logit, np.nan), d_scale=torch.full_like(k.scale, np.nan)))
            else:
                gout.append(None)
        sp.backward(kfs, scene.views, gin, gout)
        torch.cuda.synchronize()
        res["grads"] = [None if g is None else {k: v.cpu().numpy() for k, v in g.items()} for g in gout]
        if pose:
            res["pose"] = np.stack([g["pose"].cpu().numpy().reshape(3, 4) for g in gin])
    return res


def gpu_key_list(res, scene):
    """(keys, vals) of the GPU's sorted tile lists in the oracle's key format."""
    offs, ent = res["offsets"], res["entries"]
    tiles = np.repeat(np.arange(len(offs) - 1, dtype=np.uint64), np.diff(offs).astype(np.int64))
    keys = (tiles << np.uint64(32)) | (ent >> np.uint64(32))
    vals = (ent & np.uint64(0xffffffff)).astype(np.uint32)
    return keys, vals


def near_pairs(scene, o=None):
    """Per view, the set of Gaussians whose binning or key rounding is near a threshold."""
    out = []
    for k in range(len(scene.views)):
        P = oracle.project(scene, k, o)
        out.append(set(np.nonzero(P["near"])[0].tolist()))
    return out


def compare_keys(res, scene, o=None, max_aside_frac=0.01):
    """Keys and values must match the oracle's brute-force list exactly, after setting
    aside entries of (view, Gaussian) pairs with a near decision; at most max_aside_frac
    of the oracle's entries may be set aside (a margin too wide, or a bug that lands next
    to thresholds, would otherwise hide mismatches). Returns the number set aside."""
    ok, ov, onear = oracle.keys(scene, o)
    gk, gv = gpu_key_list(res, scene)
    tw, th = (o.tile_w, o.tile_h) if o is not None else (16, 16)
    counts = [((v.width + tw - 1) // tw) * ((v.height + th - 1) // th) for v in scene.views]
    tile_view = np.repeat(np.arange(len(counts)), counts)
    near = near_pairs(scene, o)

    def keep_mask(keys, vals):
        t = (keys >> np.uint64(32)).astype(np.int64)
        vw = tile_view[t]
        return np.array([int(g) not in near[int(w)] for w, g in zip(vw, vals)], bool) if len(keys) else np.zeros(0, bool)

    mo, mg = keep_mask(ok, ov), keep_mask(gk, gv)
    n_aside = int((~mo).sum())
    assert n_aside <= max_aside_frac * max(len(ok), 1), (n_aside, len(ok))
    np.testing.assert_array_equal(gk[mg], ok[mo])
    np.testing.assert_array_equal(gv[mg], ov[mo])
    return n_aside


def compare_images(res, ref, atol=IMAGE_ATOL, max_near_frac=0.01):
    """Images within atol and contributor counts exact on pixels without a near
    decision; at most max_near_frac of all pixels may be near. Returns (max error on
    clean pixels, number of near pixels)."""
    worst, n_near, n_all = 0.0, 0, 0
    base = 0
    for k, (g, r) in enumerate(zip(res["images"], ref)):
        clean = r["near"] == 0
        n_near += int((~clean).sum())
        n_all += clean.size
        for q in ("rgb", "depth", "alpha"):
            d = np.abs(g[q].astype(np.float64) - r[q])
            d = d[:, clean] if q == "rgb" else d[clean]
            worst = max(worst, float(d.max()) if d.size else 0.0)
            assert d.size == 0 or d.max() <= atol, (k, q, float(d.max()))
        hw = r["n_contrib"].size
        nc = res["n_contrib"][base:base + hw].reshape(r["n_contrib"].shape)
        tf = res["t_final"][base:base + hw].reshape(r["n_contrib"].shape)
        np.testing.assert_array_equal(nc[clean], r["n_contrib"][clean])
        assert np.abs(tf[clean] - r["t_final"][clean]).max() <= atol
        base += hw
    assert n_near <= max_near_frac * max(n_all, 1), (n_near, n_all)
    return worst, n_near


GRAD_ABS_RTOL = 1e-4       # FP32 error per summed term, relative to the term's magnitude


def compare_grads(res, ref_grads, rtol=GRAD_RTOL, abs_rtol=GRAD_ABS_RTOL, floor=1e-6, near_ratio=2.0,
                  max_near_frac=0.1):
    """Gradients within rtol |ref| + abs_rtol A + floor max|ref|, where A is the sum of
    the magnitudes of the per-pixel contributions the oracle reports (a gradient is a sum
    over pixels and views whose terms can cancel; FP32 carries an error proportional to
    the terms, not to their sum) and the floor covers near-zero entries whose single
    contributions cancel inside the chain rule. Gaussians the oracle flags as reached by
    a near decision are held to near_ratio times that, and must be at most max_near_frac
    of all. Measured on the room crop and the uneven batching scene: flagged Gaussians
    at most 0.75 of the bound (near_ratio 2 leaves a 2.7x margin), 6.2 % and 14.9 % of
    the Gaussians flagged. Returns the worst ratio on the others (<= 1 passes).

    compare_grads.last_stats records what the cancellation allowance admits: of the
    entries not flagged near, how many exceed the plain bound rtol |ref| + floor max|ref|
    (n_plain_fail, of n_entries), the largest A / |ref| among those (cancellation factor)
    and their worst ratio to the plain bound; and the near-flagged Gaussians (n_flagged
    of n_gaussians) with their worst ratio to the full bound."""
    worst, n_flag, n_all = 0.0, 0, 0
    n_entries, n_plain_fail, canc, plain_worst, near_worst = 0, 0, 0.0, 0.0, 0.0
    for g, r in zip(res["grads"], ref_grads):
        if g is None:
            continue
        nr = r["near"]
        n_flag += int(nr.sum())
        n_all += nr.size
        for q in ("d_offset", "d_rgb", "d_logit", "d_scale"):
            gq, rq, aq = g[q].astype(np.float64), r[q], r["abs"][q]
            assert np.all(np.isfinite(gq)), q
            err = np.abs(gq - rq)
            fl = floor * np.abs(rq).max()
            ratio = err / (rtol * np.abs(rq) + abs_rtol * aq + fl + 1e-30)
            clean = np.broadcast_to(~nr, ratio.shape)
            if clean.any():
                worst = max(worst, float(ratio[clean].max()))
                plain = err[clean] / (rtol * np.abs(rq[clean]) + fl + 1e-30)
                fail = plain > 1.0
                n_entries += int(clean.sum())
                n_plain_fail += int(fail.sum())
                if fail.any():
                    plain_worst = max(plain_worst, float(plain[fail].max()))
                    canc = max(canc, float((aq[clean][fail] / (np.abs(rq[clean][fail]) + 1e-300)).max()))
            if (~clean).any():
                near_worst = max(near_worst, float(ratio[~clean].max()))
                assert float(ratio[~clean].max()) <= near_ratio, (q, float(ratio[~clean].max()))
    assert n_flag <= max_near_frac * max(n_all, 1), (n_flag, n_all)
    compare_grads.last_flagged = n_flag
    compare_grads.last_stats = dict(n_entries=n_entries, n_plain_fail=n_plain_fail, max_cancellation=canc,
                                    plain_worst=plain_worst, n_flagged=n_flag, n_gaussians=n_all,
                                    near_worst=near_worst)
    return worst


def grad_stats_line(tag):
    """One printed line of compare_grads.last_stats (read from the test log)."""
    s = compare_grads.last_stats
    return ("%s: grads %d entries, %d over the plain bound (worst %.2f of it, A/|ref| up to %.3g); "
            "near-flagged %d of %d Gaussians (worst %.2f of the full bound)" %
            (tag, s["n_entries"], s["n_plain_fail"], s["plain_worst"], s["max_cancellation"], s["n_flagged"],
             s["n_gaussians"], s["near_worst"]))


def l1_grads(scene, renders):
    loss, g = oracle.l1_loss(scene, renders)
    return loss, [dict(rgb=x["rgb"].astype(np.float32), depth=x["depth"].astype(np.float32)) for x in g]


def compare_pose(res, ref, absum, rtol=GRAD_RTOL, abs_rtol=GRAD_ABS_RTOL, floor=1e-6):
    """View-pose gradients within rtol |ref| + abs_rtol A + floor max|ref| (A: the
    oracle's sum of per-pixel contribution magnitudes). Returns the worst ratio."""
    g = res["pose"].astype(np.float64)
    assert np.all(np.isfinite(g))
    ratio = np.abs(g - ref) / (rtol * np.abs(ref) + abs_rtol * absum + floor * np.abs(ref).max() + 1e-30)
    return float(ratio.max())
