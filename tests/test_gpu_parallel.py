"""Frame-sharded mapping on the GPU (one rank): every frame of a short sequence is mapped
by the library with its fixed neighbours, the Eq. 1 loss of each frame falls, the
neighbour Gaussians a frame renders are those of earlier waves, and the own-only mode
(each frame with its own Gaussians) maps every frame independently of the others."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def seq():
    from paper_2603_21055_gb300 import learned, parallel
    fr = learned.room_frames(31, n_frames=6, size=(160, 120, 150.0, 80.0, 60.0))
    return parallel.Sequence(fr["poses"], fr["rgb"], fr["obs"], (160, 120, 150.0, 80.0, 60.0))


@pytest.mark.parametrize("own_only,views", [(False, "all"), (True, "all"), (False, "one")])
def test_sequence_mapping_one_rank(seq, own_only, views):
    import torch
    from paper_2603_21055_gb300 import parallel
    fm = parallel.FrameMapper(seq, nn=2, iters=30, views_per_iter=views)
    sm = parallel.ShardedMapping(seq.n_frames, seq.hw, fm, own_only=own_only)
    params = sm.run()
    assert sorted(params) == list(range(seq.n_frames))
    for i in range(seq.n_frames):
        first, last = fm.losses[i]
        assert np.isfinite(first) and last < 0.9 * first, (i, first, last)
        # one rank: waves of one frame, so every earlier neighbour is mapped and fixed
        assert fm.n_keyframes[i] == (1 if own_only else 1 + min(2, i))
        p = params[i]
        assert torch.isfinite(p).all()
        off, rgb, lg, sc = parallel.split_params(p, 120, 160)
        assert (sc > 0).all()
        assert off.abs().max().item() > 0           # the offsets moved
        assert fm.psnr[i] > 20.0
    # the stored parameters are the learnable ones the last iteration left
    init = parallel.plain_init(seq, 0, "cuda")
    assert not torch.equal(init, params[0])
