"""The device-side pieces of the rendering-based camera initialisation (Sec. 3.3,
"Initialization"): a keyframe world transform read from device memory renders what the
equivalent moved view renders; the silhouette-masked L1 loss; the pose update
(sgad_pose_adam_step) against the host definition (twist gradient, Adam, exp of the
twist); and PoseRefiner.step without any host synchronisation."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _rigid(rng, ang, trans):
    from paper_2603_21055_gb300.synth import random_unit, rotation_about
    return np.concatenate([rotation_about(random_unit(rng), ang), trans * random_unit(rng)[:, None]], 1)


def _compose(A, B):
    """A B of two 3x4 rigid transforms (as 4x4)."""
    return np.concatenate([A[:, :3] @ B[:, :3], (A[:, :3] @ B[:, 3] + A[:, 3])[:, None]], 1)


def test_world_transform_equals_moved_view(scene1):
    """Centres moved by M on the device, seen by W, against the centres seen by W M."""
    import torch
    from paper_2603_21055_gb300 import splat, synth
    rng = np.random.default_rng(3)
    M = _rigid(rng, math.radians(1.5), 0.02)
    k = scene1.keyframes[0]
    v = scene1.views[0]
    W = np.asarray(v.pose, np.float64)
    WM = synth._f32pose(_compose(W, M.astype(np.float32).astype(np.float64)))
    fixed = synth.Keyframe(k.cam, k.depth, k.offset, k.rgb, k.logit, k.scale, learnable=False)
    kfs = splat.upload_keyframes(synth.Scene([fixed], [v], scene1.target_rgb, scene1.target_depth))
    out = []
    for tr, view in ((torch.as_tensor(M.astype(np.float32).reshape(12)).cuda(), v),
                     (None, synth.Camera(v.width, v.height, v.fx, v.fy, v.cx, v.cy, WM))):
        kk = [splat.DeviceKeyframe(kf.cam, kf.depth, kf.offset, kf.rgb, kf.logit, kf.scale, False, world_transform=tr)
              for kf in kfs]
        sp = splat.Splatter()
        sp.plan(kk, [view])
        ims = splat.alloc_images([view])
        sp.forward(kk, [view], ims)
        assert sp.check()[0] == 0
        out.append({q: t.cpu().numpy() for q, t in ims[0].items()})
    for q in ("rgb", "depth", "alpha"):
        d = np.abs(out[0][q] - out[1][q])
        # FP32 evaluation orders differ (W (M mu) against (W M) mu): equal to rounding,
        # except where an alpha or stop decision flips
        assert np.quantile(d, 0.99) <= 1e-4 and d.mean() <= 1e-5, (q, float(np.quantile(d, 0.99)), float(d.mean()))


def test_world_transform_needs_a_fixed_keyframe(scene1):
    import ctypes as C
    from paper_2603_21055_gb300 import binding as B
    from paper_2603_21055_gb300 import splat
    import torch
    kfs = splat.upload_keyframes(scene1)
    kfs[0].world_transform = torch.zeros(12, device="cuda")
    sp = splat.Splatter()
    ka, va = sp.kf_structs(kfs), sp.view_structs(scene1.views)
    n = C.c_size_t(0)
    assert B.load().sgad_workspace_size(sp.ctx, ka, 1, va, 1, 0, C.byref(n)) == B.SGAD_ERR_INVALID_ARG


def test_silhouette_masked_l1(scene1):
    """Pixels whose rendered alpha is at most min_alpha add no loss and get zero
    gradients; the others keep the unmasked values."""
    import torch
    from paper_2603_21055_gb300 import splat
    sp = splat.Splatter()
    kfs = splat.upload_keyframes(scene1)
    sp.plan(kfs, scene1.views)
    ims = splat.alloc_images(scene1.views)
    sp.forward(kfs, scene1.views, ims)
    trgb, tdep = splat.upload_targets(scene1)
    tdep = [torch.full_like(ims[0]["depth"], 1.5)]
    res = []
    for thr in (-1.0, 0.99):
        d_rgb, d_dep = [torch.empty_like(ims[0]["rgb"])], [torch.empty_like(ims[0]["depth"])]
        loss, valid = torch.zeros(1, device="cuda"), torch.zeros(1, dtype=torch.int32, device="cuda")
        sp.l1_loss_grad(scene1.views, ims, trgb, tdep, 0.8, 0.5, d_rgb, d_dep, loss, valid, min_alpha=thr)
        res.append((d_rgb[0].cpu().numpy(), d_dep[0].cpu().numpy(), float(loss.item())))
    keep = ims[0]["alpha"].cpu().numpy() > 0.99
    assert 0 < keep.sum() < keep.size
    np.testing.assert_array_equal(res[1][0][:, keep], res[0][0][:, keep])
    np.testing.assert_array_equal(res[1][1][keep], res[0][1][keep])
    assert not res[1][0][:, ~keep].any() and not res[1][1][~keep].any()
    hw = keep.size
    r = ims[0]["rgb"].cpu().numpy().astype(np.float64)
    ref = 0.8 * (np.abs(r - trgb[0].cpu().numpy())[:, keep].sum() / (3 * hw)) + \
        0.5 * (np.abs(ims[0]["depth"].cpu().numpy().astype(np.float64) - 1.5)[keep].sum() / hw)
    assert abs(res[1][2] - ref) <= 1e-5 * ref


def test_pose_adam_step_matches_the_host_definition():
    """Two steps of sgad_pose_adam_step against the host twist gradient, Adam and twist
    exponential, with M = W0^-1 E W0 and the pose E W0."""
    import torch
    from paper_2603_21055_gb300 import binding as B
    from paper_2603_21055_gb300.synth import pose_inverse
    from paper_2603_21055_gb300.tracking import exp_twist, twist_gradient
    rng = np.random.default_rng(4)
    W0 = _rigid(rng, 0.8, 1.0).astype(np.float32)
    st = torch.zeros(B.SGAD_POSE_STATE_FLOATS, device="cuda")
    eye = np.array([1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0], np.float32)
    st[0:12] = torch.as_tensor(eye)
    st[12:24] = torch.as_tensor(eye)
    E = np.eye(4)
    m, v = np.zeros(6), np.zeros(6)
    lr = np.array([3e-3] * 3 + [2e-3] * 3)
    W0d = W0.astype(np.float64)
    for n in (1, 2):
        dp = rng.normal(size=12).astype(np.float32)
        dpt = torch.as_tensor(dp).cuda()
        B.sgad_pose_adam_step(dpt.data_ptr(), W0.reshape(12), st.data_ptr(), 3e-3, 2e-3, 0.9, 0.999, 1e-12,
                              torch.cuda.current_stream().cuda_stream)
        g = twist_gradient(W0d, dp.astype(np.float64))
        m = 0.9 * m + 0.1 * g
        v = 0.999 * v + 0.001 * g * g
        xi = -lr * (m / (1 - 0.9 ** n)) / (np.sqrt(v / (1 - 0.999 ** n)) + 1e-12)
        E = exp_twist(xi) @ E
    s = st.cpu().numpy().astype(np.float64)
    W04 = np.vstack([W0d, [0, 0, 0, 1]])
    Minv = np.vstack([pose_inverse(W0d), [0, 0, 0, 1]])
    np.testing.assert_allclose(s[0:12].reshape(3, 4), E[:3], atol=2e-6)
    np.testing.assert_allclose(s[12:24].reshape(3, 4), (Minv @ E @ W04)[:3], atol=2e-6)
    np.testing.assert_allclose(s[37:49].reshape(3, 4), (E @ W04)[:3], atol=2e-6)
    assert s[36] == 2.0


def test_pose_refiner_step_does_not_synchronise(scene1):
    """PoseRefiner.step issues library launches and device tensor operations only: under
    torch's synchronisation check in error mode it runs without raising."""
    import torch
    from paper_2603_21055_gb300 import splat, synth
    from paper_2603_21055_gb300.tracking import PoseRefiner
    k = scene1.keyframes[0]
    fixed = synth.Keyframe(k.cam, k.depth, k.offset, k.rgb, k.logit, k.scale, learnable=False)
    kfs = splat.upload_keyframes(synth.Scene([fixed], scene1.views, scene1.target_rgb, scene1.target_depth))
    trgb, _ = splat.upload_targets(scene1)
    pr = PoseRefiner(kfs, scene1.views[0], trgb[0], torch.full_like(trgb[0][0], 1.5))
    torch.cuda.synchronize()
    torch.cuda.set_sync_debug_mode("error")
    try:
        for _ in range(5):
            pr.step()
    finally:
        torch.cuda.set_sync_debug_mode("default")
    assert len(pr.history) == 5 and np.all(np.isfinite(pr.history))
    assert np.all(np.isfinite(pr.pose))
