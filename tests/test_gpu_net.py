"""GPU parity of the proposal net's tensor-core kernels against the FP64 oracle.

Every layer is checked on the GPU's own bf16 inputs (so the comparison isolates one
kernel): a bf16 output may differ from the FP64 value by its rounding (2^-8 relative)
plus the FP32 accumulation error, bounded by 1e-5 times the sum of the magnitudes of
the summed products (A below); FP32 outputs and parameter gradients (long sums over
pixels, accumulated with atomics) by 1e-4 A. Sizes: two frames of 5 x 150 pixels, so
each image row spans a full 128-pixel tile and a ragged 22-pixel one (the weight
gradient's 128-pixel K blocks the same); and two frames of 240 x 630 pixels (2,400 row
tiles of 128 pixels, the last of each row ragged, and as many weight-gradient K blocks),
several times the persistent grids, so that every block of the convolutions
walks its three-stage TMA ring and flips its double TMEM accumulator many times and every
weight-gradient block cycles through its three load stages.
"""
import numpy as np
import pytest

from oracle import net as onet

pytestmark = pytest.mark.gpu

SIZES = {"5x150": (2, 5, 150), "240x630": (2, 240, 630)}


def _bf(t):
    return t.float().cpu().numpy().astype(np.float64)


@pytest.fixture(scope="module", params=sorted(SIZES))
def run(request):
    import torch
    N, H, W = SIZES[request.param]
    from paper_2603_21055_gb300.proposal import ProposalNet
    rng = np.random.default_rng(11)
    params = [(w, rng.normal(0, 0.05, size=b.shape).astype(np.float32)) for w, b in onet.init_params(3)]
    net = ProposalNet(params)
    rgb = torch.as_tensor(rng.uniform(size=(N, 3, H, W)).astype(np.float32)).cuda()
    depth = torch.as_tensor(rng.uniform(0.5, 4.0, size=(N, H, W)).astype(np.float32)).cuda()
    td = torch.as_tensor(rng.normal(0, 0.01, size=(N, H, W)).astype(np.float32)).cuda()
    tl = torch.as_tensor(rng.normal(1, 0.5, size=(N, H, W)).astype(np.float32)).cuda()
    delta = torch.full((N, H, W), float("nan"), device="cuda")
    logit = torch.full((N, H, W), float("nan"), device="cuda")
    net.forward(rgb, depth, delta, logit)
    net.loss_grad(td, tl, logit_weight=0.5)
    net.backward()
    torch.cuda.synchronize()
    assert net.check() == 0
    bufs = net.buffers()
    npx = N * H * W

    def planar(ptr, c):
        # chunk-planar units [frame][row][chunk][pixel] of 8 channels -> (N, H, W, c)
        a = _bf(net.workspace_array(ptr, npx * c)).reshape(N, H, c // 8, W, 8)
        return a.transpose(0, 1, 3, 2, 4).reshape(N, H, W, c)

    x = [planar(bufs.x[0], 16)] + [planar(bufs.x[l], 32) for l in (1, 2, 3)]
    y4 = net.workspace_array(bufs.y4, npx * 2, torch.float32).cpu().numpy().astype(np.float64).reshape(N, H, W, 2)
    dy4 = planar(bufs.dy4, 16)
    dpre = [planar(bufs.dpre[l], 32) for l in range(3)]
    return dict(net=net, params=params, rgb=rgb.cpu().numpy(), depth=depth.cpu().numpy(), td=td.cpu().numpy(),
                tl=tl.cpu().numpy(), delta=delta.cpu().numpy(), logit=logit.cpu().numpy(), x=x, y4=y4, dy4=dy4,
                dpre=dpre, dw=[t.cpu().numpy().astype(np.float64) for t in net.dw],
                db=[t.cpu().numpy().astype(np.float64) for t in net.db], loss=float(net.loss.item()))


def _wq(params, l):
    """bf16 weights of layer l in the oracle layout (3, 3, cin, cout)."""
    return onet.bf16(params[l][0])


def _abs_conv(x, w):
    return onet.conv3x3(np.abs(x), np.abs(w), np.zeros(w.shape[3]))


def test_input_packing_exact(run):
    ref = onet.pack_input(run["rgb"], run["depth"])
    np.testing.assert_array_equal(run["x"][0][..., :4], ref)
    assert np.all(run["x"][0][..., 4:] == 0.0)


@pytest.mark.parametrize("l", [0, 1, 2])
def test_conv_forward_layers(run, l):
    xin = run["x"][l][..., :onet.CHANNELS[l]]
    w = _wq(run["params"], l)
    b = run["params"][l][1].astype(np.float64)
    ref = np.maximum(onet.conv3x3(xin, w, b), 0.0)
    A = _abs_conv(xin, w) + np.abs(b)
    got = run["x"][l + 1]
    err = np.abs(got - ref)
    assert np.all(err <= 2.0 ** -8 * np.abs(ref) + 1e-5 * A + 1e-30), float((err / (2.0 ** -8 * np.abs(ref) + 1e-5 * A + 1e-30)).max())


def test_conv_output_layer(run):
    xin = run["x"][3]
    w = _wq(run["params"], 3)
    b = run["params"][3][1].astype(np.float64)
    ref = onet.conv3x3(xin, w, b)
    A = _abs_conv(xin, w) + np.abs(b)
    assert np.all(np.abs(run["y4"] - ref) <= 1e-5 * A)
    np.testing.assert_allclose(run["delta"], 0.01 * run["y4"][..., 0].astype(np.float32), rtol=1e-6, atol=1e-9)
    np.testing.assert_array_equal(run["logit"], run["y4"][..., 1].astype(np.float32))


def test_loss_and_output_gradient(run):
    loss, d = onet.mse_loss(run["y4"], run["td"], run["tl"], weight_logit=0.5)
    assert abs(run["loss"] - loss) <= 1e-5 * abs(loss)
    assert np.all(np.abs(run["dy4"][..., :2] - d) <= 2.0 ** -8 * np.abs(d) + 1e-12)
    assert np.all(run["dy4"][..., 2:] == 0.0)


@pytest.mark.parametrize("l", [3, 2, 1])
def test_input_gradient_layers(run, l):
    """dpre[l-1] = (W_l^T * dy_l) [x_l > 0], on the GPU's bf16 dy_l and x_l."""
    dy = run["dy4"][..., :2] if l == 3 else run["dpre"][l]
    w = _wq(run["params"], l)
    xin = run["x"][l]
    dx, _, _ = onet.conv3x3_backward(xin, w, dy)
    ref = dx * (xin > 0)
    A = np.zeros_like(ref)
    dxa, _, _ = onet.conv3x3_backward(xin, np.abs(w), np.abs(dy))
    A = dxa
    got = run["dpre"][l - 1]
    err = np.abs(got - ref)
    bound = 2.0 ** -8 * np.abs(ref) + 1e-5 * A + 1e-30
    assert np.all(err <= bound), float((err / bound).max())


@pytest.mark.parametrize("l", [0, 1, 2, 3])
def test_weight_and_bias_gradients(run, l):
    cin, cout = onet.CHANNELS[l], onet.CHANNELS[l + 1]
    dy = run["dy4"][..., :2] if l == 3 else run["dpre"][l]
    xin = run["x"][l][..., :cin]
    _, dw, db = onet.conv3x3_backward(xin, _wq(run["params"], l), dy)
    _, dwa, dba = onet.conv3x3_backward(np.abs(xin), np.abs(_wq(run["params"], l)), np.abs(dy))
    got_w = run["dw"][l][:, :cin, :cout].reshape(3, 3, cin, cout)
    got_b = run["db"][l][:cout]
    assert np.all(np.abs(got_w - dw) <= 1e-4 * dwa + 1e-30), float(np.abs(got_w - dw).max())
    assert np.all(np.abs(got_b - db) <= 1e-4 * dba + 1e-30)
    # padded rows and columns stay exactly zero
    full = run["dw"][l]
    mask = np.ones(full.shape, bool)
    mask[:, :cin, :cout] = False
    assert np.all(full[mask] == 0.0)


def test_training_reduces_loss():
    """A few Adam steps on one fixed batch lower the training loss (GPU end to end)."""
    import torch
    from paper_2603_21055_gb300.proposal import ProposalNet
    rng = np.random.default_rng(12)
    net = ProposalNet(seed=5)
    rgb = torch.as_tensor(rng.uniform(size=(2, 3, 24, 200)).astype(np.float32)).cuda()
    depth = torch.as_tensor(rng.uniform(0.5, 4.0, size=(2, 24, 200)).astype(np.float32)).cuda()
    td = torch.as_tensor((0.01 * (depth.cpu().numpy() - 2.0)).astype(np.float32)).cuda()
    tl = torch.as_tensor(np.full((2, 24, 200), 2.0, np.float32)).cuda()
    losses = []
    for _ in range(60):
        net.train_step(rgb, depth, td, tl)
        losses.append(float(net.loss.item()))
    assert net.check() == 0
    assert losses[-1] < 0.2 * losses[0], (losses[0], losses[-1])
