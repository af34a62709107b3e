"""Host-side checks of the learned-initialisation data: observed depth is the ray-cast
depth plus ~1 cm noise on a 2 mm grid; windows tile the frames; a window's scene has
every frame as a learnable keyframe with the plain initialisation, fitted against the
4 neighbour views halfway between consecutive frames."""
import numpy as np

from paper_2603_21055_gb300 import learned, synth

SMALL = (80, 60, 75.0, 40.0, 30.0)


def test_observed_depth_noise_and_quantisation():
    fr = learned.room_frames(3, n_frames=3, size=SMALL)
    q = fr["obs"] / learned.DEPTH_QUANT
    assert np.all(np.abs(q - np.round(q)) < 1e-3)
    e = (fr["obs"] - fr["depth"]).astype(np.float64)
    assert 0.008 < e.std() < 0.012 and abs(e.mean()) < 1e-3
    assert fr["rgb"].min() >= 0.0 and fr["rgb"].max() <= 1.0


def test_midpoint_pose():
    """Halfway between two poses: the rotation is turned by half the relative rotation
    (composing the half turn twice gives the full one) and the position is the mean."""
    rng = np.random.default_rng(0)
    a = np.concatenate([synth.rotation_about(rng.normal(size=3), 0.4), rng.normal(size=(3, 1))], 1)
    b = np.concatenate([a[:, :3] @ synth.rotation_about(rng.normal(size=3), 0.2), rng.normal(size=(3, 1))], 1)
    m = learned.midpoint_pose(a, b)
    half = a[:, :3].T @ m[:, :3]
    np.testing.assert_allclose(half @ half, a[:, :3].T @ b[:, :3], atol=1e-12)
    np.testing.assert_allclose(m[:, 3], 0.5 * (a[:, 3] + b[:, 3]), atol=1e-15)
    np.testing.assert_allclose(m[:, :3] @ m[:, :3].T, np.eye(3), atol=1e-12)
    np.testing.assert_allclose(learned.midpoint_pose(a, a), a, atol=1e-12)


def test_windows_and_scene():
    assert learned.windows(12) == [[0, 1, 2, 3, 4], [5, 6, 7, 8, 9]]
    fr = learned.room_frames(4, n_frames=5, size=SMALL)
    assert fr["mid_poses"].shape[0] == 4 and fr["mid_obs"].shape == (4, 60, 80)
    sc = learned.window_scene(fr, [0, 1, 2, 3, 4])
    assert len(sc.keyframes) == 5 and len(sc.views) == 4
    for k, i in zip(sc.keyframes, range(5)):
        assert k.learnable and np.all(k.offset == 0) and np.all(k.logit == learned.PLAIN_LOGIT)
        np.testing.assert_allclose(k.scale, fr["obs"][i] / 75.0, rtol=1e-6)
    for v, i in zip(sc.views, range(4)):
        # the view is the midpoint pose between frames i and i + 1 (world->cam of it)
        c2w = np.vstack([learned.midpoint_pose(fr["poses"][i].astype(np.float64),
                                               fr["poses"][i + 1].astype(np.float64)), [0, 0, 0, 1]])
        w2c = np.vstack([v.pose.astype(np.float64), [0, 0, 0, 1]])
        np.testing.assert_allclose(w2c @ c2w, np.eye(4), atol=1e-5)
        np.testing.assert_array_equal(sc.target_rgb[i], fr["mid_rgb"][i])
        np.testing.assert_array_equal(sc.target_depth[i], fr["mid_obs"][i])
    assert sc.rgb_weight == learned.RGB_WEIGHT and sc.depth_weight == learned.DEPTH_WEIGHT
