"""Rendering-based camera initialisation on the GPU: starting from the previous frame's
pose, descending d loss / d pose of the (silhouette-masked) rendering error of the
previous frame's Gaussians against the new frame (2 cm and 1 degree away) must reach the
objective's value at the true pose and bring the estimate closer to it."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _pose_errors(W, W_true):
    R, Rt = W[:, :3], W_true[:, :3]
    ang = np.degrees(np.arccos(np.clip((np.trace(R @ Rt.T) - 1) / 2, -1, 1)))
    # camera centres: c = -R^T t
    c, ct = -R.T @ W[:, 3], -Rt.T @ W_true[:, 3]
    return float(np.linalg.norm(c - ct)), float(ang)


def test_pose_refinement_recovers_the_new_frame():
    import torch
    from paper_2603_21055_gb300 import splat, synth
    from paper_2603_21055_gb300.tracking import PoseRefiner
    w, h, f, cx, cy = 320, 240, 300.0, 160.0, 120.0
    rng = np.random.default_rng(21)
    centre = np.array([3.0, 2.5, 1.5])
    room = synth.make_room(rng, keep_free=(centre, 1.1))
    prev = synth.keyframe_path(rng, 1, centre)[0]                    # previous frame, cam -> world
    # the new frame: 2 cm along a seeded direction and 1 degree about a seeded axis
    d = synth.random_unit(rng)
    cur = prev.copy()
    cur[:, :3] = synth.rotation_about(synth.random_unit(rng), np.radians(1.0)) @ prev[:, :3]
    cur[:, 3] = prev[:, 3] + 0.02 * d
    dep, rgb = synth.raycast(room, prev, w, h, f, f, cx, cy)
    tdep, trgb = synth.raycast(room, cur, w, h, f, f, cx, cy)
    # the previous frame's Gaussians as mapping leaves them: opaque and sharp
    logit = np.full((h, w), 6.0, np.float32)
    kf = synth.Keyframe(synth.Camera(w, h, f, f, cx, cy, synth._f32pose(prev)), dep, np.zeros_like(dep), rgb, logit,
                        (0.5 * dep / np.float32(f)).astype(np.float32), False)
    kfs = splat.upload_keyframes(synth.Scene([kf], [], [], [], 1.0))
    true_w2c = synth.pose_inverse(cur)
    start = synth._f32pose(synth.pose_inverse(prev))
    cam0 = synth.Camera(w, h, f, f, cx, cy, start)
    pr = PoseRefiner(kfs, cam0, torch.as_tensor(trgb).cuda(), torch.as_tensor(tdep).cuda())
    e0 = _pose_errors(np.asarray(start, np.float64), true_w2c)
    pr.run(200)
    e1 = _pose_errors(pr.pose, true_w2c)
    # the objective's value at the true pose (one evaluation there)
    at_true = PoseRefiner(kfs, synth.Camera(w, h, f, f, cx, cy, synth._f32pose(true_w2c)),
                          torch.as_tensor(trgb).cuda(), torch.as_tensor(tdep).cuda())
    l_true = at_true.step()
    print("pose error: %.4f m %.3f deg -> %.4f m %.3f deg; loss %.4f -> %.4f (at the true pose %.4f)"
          % (e0 + e1 + (pr.history[0], pr.history[-1], l_true)))
    # the descent reaches the objective's level at the true pose, and the pose errors
    # shrink (what is left is the offset of this objective's minimum: the previous frame's
    # Gaussians render a slightly blurred image)
    assert pr.history[-1] <= 1.05 * l_true
    assert e1[1] < 0.5 * e0[1] and e1[0] < 0.75 * e0[0]
