"""The learned-initialisation pipeline on small frames (GPU): plain-mapping targets,
training the net on them, the gain of the trained net over the plain initialisation on
held-out rooms, and the plain initialisation as fallback when the net's prediction
renders worse."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SMALL = (160, 120, 150.0, 80.0, 60.0)
FRAMES = 10


@pytest.fixture(scope="module")
def trained():
    """A net trained on the plain-converged offsets and logits of 6 rooms (12 windows)."""
    import torch
    from paper_2603_21055_gb300 import learned
    from paper_2603_21055_gb300.proposal import ProposalNet
    ds = learned.Dataset(6 * FRAMES, size=SMALL)
    for seed in range(100, 106):
        fr = learned.room_frames(seed, n_frames=FRAMES, size=SMALL)
        for idx in learned.windows(FRAMES):
            offs, lgs = learned.plain_targets(fr, idx, iters=100)
            for j, i in enumerate(idx):
                assert torch.isfinite(offs[j]).all() and torch.isfinite(lgs[j]).all()
                ds.add(fr["rgb"][i], fr["obs"][i], offs[j], lgs[j])
    # the plain mapping moves offsets and logits away from the initialisation
    assert float(ds.td.abs().mean()) > 1e-4 and float((ds.tl - learned.PLAIN_LOGIT).abs().mean()) > 1e-2
    net = ProposalNet(seed=1)
    curve = learned.train(net, ds, steps=600, batch=8, lr=2e-3, log=None)
    assert net.check() == 0
    assert curve[-1][1] < 0.5 * curve[0][1]
    return net


def test_trained_net_reaches_the_target_in_fewer_iterations(trained):
    """On 4 windows of 2 held-out rooms, the learned initialisation (net inference, then
    the best of the prediction, zero offsets with predicted opacities and the plain
    initialisation by first-render loss) reaches the plain arm's final PSNR - 0.5 dB in
    fewer mapping iterations on average, starts from a better first render, and uses the
    net's output on most windows."""
    from paper_2603_21055_gb300 import learned
    it_p, it_l, first_p, first_l, kept = [], [], [], [], 0
    for seed in (900, 901):
        fr = learned.room_frames(seed, n_frames=FRAMES, size=SMALL)
        for idx in learned.windows(FRAMES):
            plain = learned.time_to_psnr(fr, idx, iters=100)
            lrn = learned.time_to_psnr(fr, idx, net=trained, iters=100)
            assert plain["capacity_ok"] and lrn["capacity_ok"]
            assert np.all(np.isfinite(plain["psnr"])) and np.all(np.isfinite(lrn["psnr"]))
            assert plain["psnr"][-1] > plain["psnr"][0]          # mapping improves the fit
            target = float(plain["psnr"][-1]) - 0.5
            _, ip = learned.seconds_to(plain["psnr"], plain["times"], target)
            _, il = learned.seconds_to(lrn["psnr"], lrn["times"], target)
            it_p.append(ip)
            it_l.append(il if il is not None else 101)
            first_p.append(float(plain["psnr"][0]))
            first_l.append(float(lrn["psnr"][0]))
            kept += int(lrn["kept"] != 2)
    print("iterations to plain final - 0.5 dB: plain %s, learned %s; first render %.2f vs %.2f dB; kept %d/%d" %
          (it_p, it_l, np.mean(first_p), np.mean(first_l), kept, len(it_p)))
    assert kept >= len(it_p) - 1
    assert np.mean(first_l) > np.mean(first_p)
    assert np.mean(it_l) < np.mean(it_p)


def test_plain_initialisation_is_kept_when_the_prediction_renders_worse(trained):
    """A net whose depth-offset output is pushed 3 m off and whose opacity logits are -20:
    both initialisations built on its output render worse than the plain one, so the
    learned arm falls back to the plain initialisation and maps exactly like the plain
    arm."""
    import torch
    from paper_2603_21055_gb300 import learned
    from paper_2603_21055_gb300.proposal import ProposalNet
    bad = ProposalNet(seed=1)
    with torch.no_grad():
        for w, b in zip(bad.w, bad.b):
            w.zero_()
            b.zero_()
        bad.b[-1][0] = 300.0                 # delta = 0.01 x 300 = 3 m everywhere
        bad.b[-1][1] = -20.0                 # opacity ~2e-9: nothing renders
    fr = learned.room_frames(902, n_frames=5, size=SMALL)
    plain = learned.time_to_psnr(fr, [0, 1, 2, 3, 4], iters=20)
    lrn = learned.time_to_psnr(fr, [0, 1, 2, 3, 4], net=bad, iters=20)
    assert lrn["kept"] == 2
    assert float(lrn["predicted"][0].mean()) > 2.9
    # the same mapping up to the order of the backward's floating-point atomic additions
    np.testing.assert_allclose(lrn["psnr"][:5], plain["psnr"][:5], rtol=0, atol=1e-4)
    np.testing.assert_allclose(lrn["psnr"], plain["psnr"], rtol=0, atol=1e-2)
