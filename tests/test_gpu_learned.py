"""The learned-initialisation pipeline end to end on small frames (GPU): plain-mapping
targets, training the net on them, and both arms of the seconds-to-PSNR comparison."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SMALL = (160, 120, 150.0, 80.0, 60.0)


def test_pipeline_small():
    import torch
    from paper_2603_21055_gb300 import learned
    from paper_2603_21055_gb300.proposal import ProposalNet
    fr = learned.room_frames(7, n_frames=10, size=SMALL)
    ds = learned.Dataset(10, size=SMALL)
    for idx in learned.windows(10):
        offs, lgs = learned.plain_targets(fr, idx, iters=30)
        for j, i in enumerate(idx):
            assert torch.isfinite(offs[j]).all() and torch.isfinite(lgs[j]).all()
            ds.add(fr["rgb"][i], fr["obs"][i], offs[j], lgs[j])
    # the plain mapping moves offsets and logits away from the initialisation
    assert float(ds.td.abs().mean()) > 1e-4 and float((ds.tl - learned.PLAIN_LOGIT).abs().mean()) > 1e-2
    net = ProposalNet(seed=1)
    curve = learned.train(net, ds, steps=120, batch=4, lr=2e-3, log=None)
    assert net.check() == 0
    assert curve[-1][1] < curve[0][1]
    plain = learned.time_to_psnr(fr, [0, 1, 2, 3, 4], iters=30, target_db=20.0)
    lrn = learned.time_to_psnr(fr, [0, 1, 2, 3, 4], net=net, iters=30, target_db=20.0)
    for r in (plain, lrn):
        assert np.all(np.isfinite(r["psnr"])) and r["capacity_ok"]
    assert plain["psnr"][-1] > plain["psnr"][0]          # mapping improves the fit
    assert lrn["predicted"] is not None and plain["predicted"] is None
