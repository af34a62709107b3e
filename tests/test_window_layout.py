"""Host-side layout of splat.upload_window (CPU tensors): every array of the window is a
256-byte aligned view of one flat buffer with the scene's values, and the updated state
(offset, colour, logit, scale of every keyframe, then the loss) is its prefix."""
import numpy as np


def test_window_layout():
    import torch
    from paper_2603_21055_gb300 import splat, synth
    from paper_2603_21055_gb300.synth import crop_scene
    sc = crop_scene(synth.config1_plane(), (3, 5, 37, 21), (0, 0, 45, 31))      # odd sizes: padding needed
    buf, n_state, kfs, trgb, tdep, loss = splat.upload_window(sc, device="cpu")
    base = buf.data_ptr()
    arrays = [(kf, k) for kf, k in zip(kfs, sc.keyframes)]
    for kf, k in arrays:
        for n in ("depth", "offset", "rgb", "logit", "scale"):
            t = getattr(kf, n)
            assert (t.data_ptr() - base) % 256 == 0
            assert np.array_equal(t.numpy(), np.asarray(getattr(k, n), np.float32))
            assert t.untyped_storage().data_ptr() == buf.untyped_storage().data_ptr()
        for n in ("offset", "rgb", "logit", "scale"):
            end = (getattr(kf, n).data_ptr() - base) // 4 + getattr(kf, n).numel()
            assert end <= n_state                                      # updated arrays in the prefix
        assert (kf.depth.data_ptr() - base) // 4 >= n_state            # inputs after it
    assert (loss.data_ptr() - base) // 4 < n_state and loss.numel() == 1 and float(loss) == 0.0
    for t, a in zip(trgb + tdep, list(sc.target_rgb) + list(sc.target_depth)):
        assert (t.data_ptr() - base) % 256 == 0 and (t.data_ptr() - base) // 4 >= n_state
        assert np.array_equal(t.numpy(), np.asarray(a, np.float32))
    # no two arrays overlap
    spans = sorted(((x.data_ptr() - base) // 4, (x.data_ptr() - base) // 4 + x.numel())
                   for x in [getattr(kf, n) for kf in kfs for n in ("depth", "offset", "rgb", "logit", "scale")]
                   + trgb + tdep + [loss])
    assert all(a[1] <= b[0] for a, b in zip(spans, spans[1:]))
    assert spans[-1][1] <= buf.numel()
