"""Host-side pieces of the rendering-based camera initialisation: the projection of
d L / d W onto a left twist, checked against the definition on a synthetic objective,
and the twist exponential."""
import numpy as np

from paper_2603_21055_gb300.tracking import exp_twist, twist_gradient


def _rot(axis, ang):
    a = np.asarray(axis, float) / np.linalg.norm(axis)
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    return np.eye(3) + np.sin(ang) * K + (1 - np.cos(ang)) * K @ K


def test_twist_gradient_matches_definition():
    """L(W) = sum_g a_g . t_g with t_g = R mu_g + t: d L / d W = sum a_g (mu_g, 1)^T, and
    for W <- exp(xi) W the twist gradient is (sum t_g x a_g, sum a_g); also checked by
    central differences of L(exp(xi) W)."""
    rng = np.random.default_rng(0)
    R = _rot(rng.normal(size=3), 0.7)
    t = rng.normal(size=3)
    W = np.hstack([R, t[:, None]])
    mu = rng.normal(size=(20, 3))
    a = rng.normal(size=(20, 3))
    dW = np.zeros((3, 4))
    dW[:, :3] = a.T @ mu
    dW[:, 3] = a.sum(0)
    tg = mu @ R.T + t
    ref = np.concatenate([np.cross(tg, a).sum(0), a.sum(0)])
    np.testing.assert_allclose(twist_gradient(W, dW), ref, rtol=1e-10, atol=1e-10)

    def L(xi):
        T = exp_twist(xi) @ np.vstack([W, [0, 0, 0, 1]])
        return float(np.sum(a * (mu @ T[:3, :3].T + T[:3, 3])))
    h = 1e-6
    fd = np.array([(L(h * e) - L(-h * e)) / (2 * h) for e in np.eye(6)])
    np.testing.assert_allclose(twist_gradient(W, dW), fd, rtol=1e-6, atol=1e-6)


def test_exp_twist_is_rigid():
    rng = np.random.default_rng(1)
    for _ in range(5):
        T = exp_twist(rng.normal(size=6) * 0.3)
        np.testing.assert_allclose(T[:3, :3] @ T[:3, :3].T, np.eye(3), atol=1e-12)
        assert abs(np.linalg.det(T[:3, :3]) - 1.0) < 1e-12
    np.testing.assert_array_equal(exp_twist(np.zeros(6)), np.eye(4))
