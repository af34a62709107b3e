"""GPU parity of the SSIM term of Eq. 1 (sgad_ssim_loss_grad) against the FP64 oracle:
loss value and colour gradient, element by element, over several views of uneven sizes
(ragged 32 x 32 tiles, images narrower than the window), near-identical images (where
the gradient is a difference of large terms), the accumulate-into-d_rgb contract, a
full 640 x 480 view, and the term inside a mapping iteration.

Tolerance: the kernel works in FP32. The moments are 11 + 11 tap sums of values in
[0, 1] (relative error a few 1e-7); the variances m2 - m1^2 lose up to a factor of
m2 / C2 ~ 1e3 to cancellation, so S and the three d S / d m maps carry relative errors
up to ~1e-4, and the final blur and the 1/N scale add FP32 rounding only. Element-wise
we therefore allow 2e-3 of the largest gradient magnitude, and 1e-4 relative on the loss
(an FP32 sum of ~1e5-1e6 terms in block partials)."""
import numpy as np
import pytest

from oracle import ssim as ossim

pytestmark = pytest.mark.gpu

GRAD_TOL = 2e-3
LOSS_RTOL = 1e-4


def _cams(sizes):
    from paper_2603_21055_gb300.synth import Camera
    return [Camera(w, h, 100.0, 100.0, w / 2, h / 2, np.eye(4, dtype=np.float32)[:3].copy()) for w, h in sizes]


def _images(rng, sizes, close=False):
    xs, ys = [], []
    for w, h in sizes:
        y = rng.uniform(size=(3, h, w))
        if close:
            x = np.clip(y + rng.normal(scale=0.02, size=y.shape), 0, 1)
        else:
            # smooth structure plus noise, so windows see real (co)variances
            yy, xx = np.mgrid[0:h, 0:w]
            x = 0.5 + 0.3 * np.sin(xx[None] / 5.0 + np.arange(3)[:, None, None]) * np.cos(yy[None] / 7.0)
            x = np.clip(x + rng.normal(scale=0.1, size=y.shape), 0, 1)
        xs.append(x.astype(np.float32))
        ys.append(y.astype(np.float32))
    return xs, ys


def _run(sizes, xs, ys, weight, d_init=None):
    import torch
    from paper_2603_21055_gb300 import splat
    cams = _cams(sizes)
    sp = splat.Splatter()
    ims = [dict(rgb=torch.as_tensor(x).cuda(), depth=torch.zeros(x.shape[1:], device="cuda"),
                alpha=torch.zeros(x.shape[1:], device="cuda")) for x in xs]
    tr = [torch.as_tensor(y).cuda() for y in ys]
    d = [torch.as_tensor(di).cuda() if d_init is not None else torch.zeros_like(t)
         for di, t in zip(d_init if d_init is not None else [None] * len(tr), tr)]
    loss = torch.zeros(1, device="cuda")
    sp.ssim_loss_grad(cams, ims, tr, weight, d, loss)
    torch.cuda.synchronize()
    return loss.item(), [t.cpu().numpy().astype(np.float64) for t in d]


def _check(sizes, xs, ys, weight, got_loss, got_d, base=None):
    ref_loss = 0.0
    for k, (x, y) in enumerate(zip(xs, ys)):
        l, g = ossim.ssim_loss_grad(x.astype(np.float64), y.astype(np.float64))
        ref_loss += weight * l
        g = weight * g + (base[k] if base is not None else 0.0)
        tol = GRAD_TOL * np.abs(weight * g).max() if base is None else GRAD_TOL * np.abs(g - base[k]).max()
        err = np.abs(got_d[k] - g).max()
        assert err <= tol, (k, sizes[k], err, tol)
    assert abs(got_loss - ref_loss) <= LOSS_RTOL * abs(ref_loss), (got_loss, ref_loss)


@pytest.mark.parametrize("close", [False, True])
def test_ssim_uneven_views_match_oracle(close):
    rng = np.random.default_rng(11 + close)
    # ragged tiles, a view narrower and shorter than the 11 x 11 window, one exactly 2 x 2
    # tiles; widths that are multiples of 4 take the 16-byte staging path, the others the
    # 4-byte one
    sizes = [(70, 45), (33, 64), (7, 5), (64, 64), (1, 1), (100, 45), (4, 3)]
    xs, ys = _images(rng, sizes, close)
    loss, d = _run(sizes, xs, ys, 0.2)
    _check(sizes, xs, ys, 0.2, loss, d)


def test_ssim_adds_into_existing_gradient():
    rng = np.random.default_rng(5)
    sizes = [(50, 40), (41, 33)]
    xs, ys = _images(rng, sizes)
    base = [rng.normal(scale=1e-4, size=(3, h, w)).astype(np.float32) for w, h in sizes]
    loss, d = _run(sizes, xs, ys, 0.7, d_init=base)
    _check(sizes, xs, ys, 0.7, loss, d, base=[b.astype(np.float64) for b in base])


def test_ssim_identical_images_zero():
    rng = np.random.default_rng(6)
    sizes = [(96, 40)]
    xs, _ = _images(rng, sizes)
    loss, d = _run(sizes, xs, [x.copy() for x in xs], 1.0)
    # L_S = 1 - mean S with S = 1 up to FP32 rounding; the gradient cancels to rounding
    assert abs(loss) < 1e-5
    assert np.abs(d[0]).max() < 1e-7


def test_ssim_full_size_view_matches_oracle():
    """One 640 x 480 view of an 8-view batch (the headline image size): all 8 views run in
    the kernel, the oracle checks views 0 and 7."""
    rng = np.random.default_rng(7)
    sizes = [(640, 480)] * 8
    xs, ys = _images(rng, sizes)
    loss, d = _run(sizes, xs, ys, 0.2)
    ref_total = 0.0
    for k in (0, 7):
        l, g = ossim.ssim_loss_grad(xs[k].astype(np.float64), ys[k].astype(np.float64))
        g = 0.2 * g
        assert np.abs(d[k] - g).max() <= GRAD_TOL * np.abs(g).max()
        ref_total += 0.2 * l
    # the other views: the loss of each is a mean of per-pixel terms in [0, 2]
    assert 0.0 < loss < 8 * 0.2 * 2.0
    assert np.isfinite(loss)


def test_mapping_iteration_with_ssim_term(room2):
    """A mapping iteration with rho = 0.8, tau = 0.2, sigma = 1.0 (the supplementary
    weights): its loss equals the L1 terms plus tau L_S of the same rendering (oracle),
    and the colour gradient handed to the adjoint is the L1 gradient plus tau dL_S/dV'."""
    import torch
    from paper_2603_21055_gb300.mapping import Mapper
    from paper_2603_21055_gb300.synth import crop_scene
    import oracle
    sc = crop_scene(room2, (200, 150, 120, 90), (190, 140, 130, 100), n_keyframes=2, n_views=2)
    sc.rgb_weight, sc.ssim_weight, sc.depth_weight = 0.8, 0.2, 1.0
    mp = Mapper(sc)
    mp.forward()
    mp.loss.zero_()
    mp.sp.l1_loss_grad(mp.views, mp.images, mp.trgb, mp.tdep, sc.rgb_weight, sc.depth_weight, mp.d_rgb, mp.d_dep,
                       mp.loss, mp.valid)
    torch.cuda.synchronize()
    l1_loss = mp.loss.item()
    l1_grad = [g.cpu().numpy().astype(np.float64) for g in mp.d_rgb]
    mp.sp.ssim_loss_grad(mp.views, mp.images, mp.trgb, sc.ssim_weight, mp.d_rgb, mp.loss)
    torch.cuda.synchronize()
    ref = 0.0
    for k in range(len(sc.views)):
        x = mp.images[k]["rgb"].cpu().numpy().astype(np.float64)
        l, g = ossim.ssim_loss_grad(x, sc.target_rgb[k].astype(np.float32).astype(np.float64))
        ref += sc.ssim_weight * l
        want = l1_grad[k] + sc.ssim_weight * g
        got = mp.d_rgb[k].cpu().numpy().astype(np.float64)
        assert np.abs(got - want).max() <= GRAD_TOL * np.abs(sc.ssim_weight * g).max()
    assert abs(mp.loss.item() - (l1_loss + ref)) <= LOSS_RTOL * (l1_loss + ref)
    # the Mapper's own iteration launches the SSIM passes too, and the loss goes down
    losses = []
    for _ in range(20):
        mp.step_eager()
        losses.append(mp.loss.item())
    torch.cuda.synchronize()
    assert losses[-1] < losses[0]
    assert mp.launches_per_step() == 4 + 1 + 2 + 2 + 1 + 1 + 2
