"""Host-side checks of the learned-initialisation data: observed depth is the ray-cast
depth plus ~1 cm noise on a 2 mm grid; windows tile the frames; a window's scene has
every frame as a learnable keyframe with the plain initialisation and a view at its own
pose."""
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


def test_windows_and_scene():
    assert learned.windows(12) == [[0, 1, 2, 3, 4], [5, 6, 7, 8, 9]]
    fr = learned.room_frames(4, n_frames=5, size=SMALL)
    sc = learned.window_scene(fr, [0, 1, 2, 3, 4])
    assert len(sc.keyframes) == 5 and len(sc.views) == 5
    for k, v, i in zip(sc.keyframes, sc.views, range(5)):
        assert k.learnable and np.all(k.offset == 0) and np.all(k.logit == learned.PLAIN_LOGIT)
        np.testing.assert_allclose(k.scale, fr["obs"][i] / 75.0, rtol=1e-6)
        # the view is the keyframe's own pose: world->cam composed with cam->world is I
        c2w = np.vstack([k.cam.pose.astype(np.float64), [0, 0, 0, 1]])
        w2c = np.vstack([v.pose.astype(np.float64), [0, 0, 0, 1]])
        np.testing.assert_allclose(w2c @ c2w, np.eye(4), atol=1e-5)
    assert sc.rgb_weight == learned.RGB_WEIGHT and sc.depth_weight == learned.DEPTH_WEIGHT
