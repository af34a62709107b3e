"""Pins of the proposal-net oracle (oracle/net.py) against things other than itself: a
library correlation, identity and shift kernels, adjointness, bfloat16 rounding of
chosen values, and central finite differences of its hand-derived adjoint."""
import numpy as np
import pytest

from oracle import net


def _rand(rng, *shape):
    return rng.normal(size=shape)


def test_conv_equals_library_correlation():
    """Each output channel is the sum over input channels of a 2-D correlation with zero
    fill (scipy.signal.correlate2d, mode 'same'), plus the bias."""
    signal = pytest.importorskip("scipy.signal")
    rng = np.random.default_rng(0)
    x = _rand(rng, 2, 7, 9, 3)
    w = _rand(rng, 3, 3, 3, 2)
    b = _rand(rng, 2)
    y = net.conv3x3(x, w, b)
    for n in range(2):
        for o in range(2):
            ref = b[o] + sum(signal.correlate2d(x[n, :, :, i], w[:, :, i, o], mode="same", boundary="fill")
                             for i in range(3))
            np.testing.assert_allclose(y[n, :, :, o], ref, rtol=1e-12, atol=1e-12)


def test_identity_and_shift_kernels():
    rng = np.random.default_rng(1)
    x = _rand(rng, 1, 5, 6, 4)
    w = np.zeros((3, 3, 4, 4))
    w[1, 1] = np.eye(4)
    np.testing.assert_array_equal(net.conv3x3(x, w, np.zeros(4)), x)
    # tap (ky, kx) = (0, 1) reads the pixel one row up: y[r] = x[r - 1], zero in row 0
    w = np.zeros((3, 3, 4, 4))
    w[0, 1] = np.eye(4)
    y = net.conv3x3(x, w, np.zeros(4))
    np.testing.assert_array_equal(y[:, 1:], x[:, :-1])
    np.testing.assert_array_equal(y[:, 0], 0.0)


def test_adjointness():
    """<conv(x), g> = <x, dx(g)> and <conv_w(x), g> = <w, dW(g)> for a bias-free conv."""
    rng = np.random.default_rng(2)
    x, w, g = _rand(rng, 2, 6, 5, 3), _rand(rng, 3, 3, 3, 4), _rand(rng, 2, 6, 5, 4)
    y = net.conv3x3(x, w, np.zeros(4))
    dx, dw, db = net.conv3x3_backward(x, w, g)
    np.testing.assert_allclose(np.sum(y * g), np.sum(x * dx), rtol=1e-12)
    np.testing.assert_allclose(np.sum(y * g), np.sum(w * dw), rtol=1e-12)
    np.testing.assert_allclose(db, g.sum(axis=(0, 1, 2)), rtol=1e-12)


def test_bf16_rounding_values():
    v = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, 1.0 + 2.0 ** -7, -2.5, 0.0, 3.0e-3], np.float32)
    r = net.bf16(v)
    # 1 + 2^-8 is half way between 1 and 1 + 2^-7: ties go to the even mantissa (1.0);
    # 1 + 3 * 2^-8 is half way between 1 + 2^-7 and 1 + 2^-6: even is 1 + 2^-6
    np.testing.assert_array_equal(r[:6], [1.0, 1.0, 1.0 + 2.0 ** -6, 1.0 + 2.0 ** -7, -2.5, 0.0])
    assert abs(r[6] - 3.0e-3) <= 2.0 ** -8 * 3.0e-3       # half a unit in the 8th bit
    rng = np.random.default_rng(3)
    a = rng.normal(size=10000).astype(np.float32)
    q = net.bf16(a)
    assert np.all(np.abs(q - a) <= 2.0 ** -8 * np.abs(a) + 1e-45)
    assert np.all(net.bf16(q) == q)        # idempotent


def _fd(f, a, idx, h=1e-6):
    ap, am = a.copy(), a.copy()
    ap[idx] += h
    am[idx] -= h
    return (f(ap) - f(am)) / (2 * h)


def test_conv_backward_finite_differences():
    rng = np.random.default_rng(4)
    x, w, b, g = _rand(rng, 1, 5, 4, 3), _rand(rng, 3, 3, 3, 2), _rand(rng, 2), _rand(rng, 1, 5, 4, 2)
    dx, dw, db = net.conv3x3_backward(x, w, g)
    loss = lambda xx, ww, bb: float(np.sum(net.conv3x3(xx, ww, bb) * g))
    for idx in [(0, 0, 0, 0), (0, 4, 3, 2), (0, 2, 1, 1)]:
        assert abs(_fd(lambda a: loss(a, w, b), x, idx) - dx[idx]) <= 1e-7 * max(1.0, abs(dx[idx]))
    for idx in [(0, 0, 0, 0), (2, 2, 2, 1), (1, 0, 1, 0)]:
        assert abs(_fd(lambda a: loss(x, a, b), w, idx) - dw[idx]) <= 1e-7 * max(1.0, abs(dw[idx]))
    for o in range(2):
        assert abs(_fd(lambda a: loss(x, w, a), b, (o,)) - db[o]) <= 1e-7 * max(1.0, abs(db[o]))


def test_net_backward_finite_differences():
    """Whole net, unrounded, MSE training loss: every parameter gradient the oracle
    derives agrees with central differences of its own forward."""
    rng = np.random.default_rng(5)
    params = [(w.astype(np.float64), rng.normal(0, 0.1, size=b.shape)) for w, b in net.init_params(7)]
    x0 = np.concatenate([rng.uniform(size=(1, 6, 5, 3)), rng.uniform(0.5, 3.0, size=(1, 6, 5, 1))], axis=-1)
    td = rng.normal(0, 0.01, size=(1, 6, 5))
    tl = rng.normal(1, 0.5, size=(1, 6, 5))

    def total(ps):
        return net.mse_loss(net.forward(x0, ps, round_points=False)[-1], td, tl)[0]

    acts = net.forward(x0, params, round_points=False)
    _, dy4 = net.mse_loss(acts[-1], td, tl)
    grads, _ = net.backward(acts, params, dy4, round_points=False)
    for l in range(4):
        w, b = params[l]
        for idx in [(1, 1, 0, 0), (0, 2, w.shape[2] - 1, w.shape[3] - 1)]:
            def f(a, l=l):
                ps = list(params)
                ps[l] = (a, params[l][1])
                return total(ps)
            fd = _fd(f, w, idx)
            assert abs(fd - grads[l][0][idx]) <= 1e-6 * max(1.0, abs(fd)), (l, idx)
        def fb(a, l=l):
            ps = list(params)
            ps[l] = (params[l][0], a)
            return total(ps)
        fd = _fd(fb, b, (0,))
        assert abs(fd - grads[l][1][0]) <= 1e-6 * max(1.0, abs(fd)), l


def test_mse_loss_gradient():
    rng = np.random.default_rng(6)
    y = rng.normal(size=(2, 3, 4, 2))
    td, tl = rng.normal(0, 0.01, size=(2, 3, 4)), rng.normal(size=(2, 3, 4))
    loss, d = net.mse_loss(y, td, tl, weight_logit=0.5)
    ref = (np.sum((y[..., 0] - td / 0.01) ** 2) + 0.5 * np.sum((y[..., 1] - tl) ** 2)) / 24
    assert abs(loss - ref) <= 1e-12 * ref
    for idx in [(0, 0, 0, 0), (1, 2, 3, 1)]:
        fd = _fd(lambda a: net.mse_loss(a, td, tl, weight_logit=0.5)[0], y, idx)
        assert abs(fd - d[idx]) <= 1e-7
