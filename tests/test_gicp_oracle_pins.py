"""Pins of the geometric-tracking oracle (oracle/gicp.py) against what the mathematics fixes:
back-projection against re-projection, the K nearest neighbours against a KD-tree, the
normal of points on a plane, the invariance of the normalised shapes to the depth scale,
the correspondence rule on a hand-made case where point-to-surface and Euclidean nearest
differ, the Gauss-Newton gradient and Hessian against central differences of Eq. 2's
cost, the recovery of a known rigid motion, and the map update's overlap rule."""
import math

import numpy as np
import pytest

from oracle import gicp as G


def _surface(rng, n=40, m=30):
    """Points of a smooth, non-planar height field seen from the camera frame."""
    u, v = np.meshgrid(np.linspace(-0.6, 0.6, n), np.linspace(-0.4, 0.4, m))
    z = 2.0 + 0.15 * np.sin(3 * u) * np.cos(4 * v) + 0.3 * u * v + 0.1 * u
    pts = np.stack([u.ravel(), v.ravel(), z.ravel()], 1)
    return (pts + rng.normal(scale=1e-3, size=pts.shape)).astype(np.float32)


def test_selection_reprojects_to_its_pixels():
    rng = np.random.default_rng(0)
    h, w, f, cx, cy = 37, 51, 40.0, 25.3, 17.9
    depth = rng.uniform(0.5, 4.0, size=(h, w)).astype(np.float32)
    depth[rng.uniform(size=(h, w)) < 0.2] = 0.0
    pts, pix = G.select_points(depth, f, f, cx, cy, 5)
    grid = [(v, u) for v in range(0, h, 5) for u in range(0, w, 5) if depth[v, u] > 0]
    assert len(pts) == len(grid) == len(pix)
    for (v, u), p, q in zip(grid, pts, pix):
        assert q == v * w + u and p[2] == depth[v, u]
        assert abs(f * p[0] / p[2] + cx - u) < 1e-4 and abs(f * p[1] / p[2] + cy - v) < 1e-4


def test_knn_matches_kdtree():
    spatial = pytest.importorskip("scipy.spatial")
    rng = np.random.default_rng(1)
    P = rng.uniform(-1, 1, size=(700, 3)).astype(np.float32)
    idx = G.knn(P, 15)
    _, ref = spatial.cKDTree(P.astype(np.float64)).query(P.astype(np.float64), k=15)
    assert (idx[:, 0] == np.arange(len(P))).all()            # itself first
    for a, b in zip(idx, ref):
        assert set(a) == set(b)


def test_plane_normal_and_shape():
    rng = np.random.default_rng(2)
    n = np.array([0.3, -0.2, 0.93])
    n /= np.linalg.norm(n)
    e1 = np.cross(n, [1, 0, 0])
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(n, e1)
    ab = rng.uniform(-0.2, 0.2, size=(300, 2))
    P = (np.array([0.1, 0.2, 2.0]) + ab[:, :1] * e1 + ab[:, 1:] * e2).astype(np.float32)
    idx = G.knn(P, 20)
    C, normal, s = G.normalised_shapes(G.covariances(P, idx))
    assert (np.abs(normal @ n) > 0.999).all()
    # the smallest normalised scale is floored at sqrt(eps), the largest is 1
    w = np.linalg.eigvalsh(C)
    assert np.allclose(w[:, 0], G.EPS, rtol=1e-3) and np.allclose(w[:, 2], 1.0)


def test_normalised_shapes_ignore_depth_scale():
    rng = np.random.default_rng(3)
    P = _surface(rng)
    idx = G.knn(P, 10)
    C1, n1, _ = G.normalised_shapes(G.covariances(P, idx))
    C2, n2, _ = G.normalised_shapes(G.covariances(P * np.float32(4.0), idx))   # exact in FP32
    np.testing.assert_allclose(C1, C2, atol=1e-9)
    assert (np.abs(np.sum(n1 * n2, 1)) > 1 - 1e-9).all()


def test_correspondence_prefers_the_surface():
    """The source point lies on map Gaussian 1's plane but closer (Euclidean) to map
    Gaussian 0, whose plane it is far from: point-to-surface picks 1; out of range, none;
    only the k_match nearest are candidates."""
    src = np.array([[0.0, 0.0, 0.0], [5.0, 5.0, 5.0]], np.float32)
    mp = np.array([[0.0, 0.0, 0.02], [0.04, 0.0, 0.0]], np.float32)
    nr = np.array([[0.0, 0.0, 1.0], [0.0, 0.0, 1.0]], np.float32)
    pose = np.hstack([np.eye(3), np.zeros((3, 1))]).astype(np.float32)
    assert list(G.correspond(src, pose, mp, nr, 0.05)) == [1, -1]
    assert list(G.correspond(src, pose, mp, nr, 0.05, k_match=1)) == [0, -1]
    # equal surface distance: the nearer one wins
    mp2 = np.array([[0.03, 0.0, 0.0], [0.01, 0.0, 0.0]], np.float32)
    assert list(G.correspond(src[:1], pose, mp2, nr, 0.05)) == [1]
    # six map points on the plane z = 0.001 at growing distance and one on z = 0 farther
    # out: the surface-exact one is the 7th nearest, outside the 5 candidates
    far = np.array([[0.005 * (k + 1), 0.0, 0.001] for k in range(6)] + [[0.04, 0.0, 0.0]], np.float32)
    nrm = np.tile(np.array([[0.0, 0.0, 1.0]], np.float32), (7, 1))
    assert list(G.correspond(src[:1], pose, far, nrm, 0.05)) == [0]
    assert list(G.correspond(src[:1], pose, far, nrm, 0.05, k_match=7)) == [6]


def _pair(rng):
    P = _surface(rng)
    src = dict(points=P)
    idx = G.knn(P, 10)
    src["cov"], src["normal"], _ = G.normalised_shapes(G.covariances(P, idx))
    return src


def test_gn_gradient_and_hessian_match_central_differences():
    rng = np.random.default_rng(4)
    src = _pair(rng)
    W = np.hstack([G.exp_so3([0.01, -0.02, 0.015]), [[0.02], [-0.01], [0.03]]])
    mp = dict(points=G.transform32(W.astype(np.float32), src["points"]),
              cov=np.einsum("ij,mjk,lk->mil", W[:, :3], src["cov"], W[:, :3]),
              normal=src["normal"] @ W[:, :3].T)
    pose = np.hstack([G.exp_so3([0.003, 0.001, -0.002]), [[0.005], [0.0], [-0.004]]])
    idx = G.correspond(src["points"], pose.astype(np.float32), mp["points"], mp["normal"], 0.05)
    assert (idx >= 0).sum() > 100
    H, g, cost, n = G.gn_system(src["points"], src["cov"], mp["points"], mp["cov"], idx, pose)

    def cost_at(base, ids, xi):
        # the covariance term held fixed at `base`, as in the linearisation
        P = G.apply_step(base, xi)
        R0 = base[:, :3]
        c = 0.0
        for i, j in enumerate(ids):
            if j < 0:
                continue
            x = P[:, :3] @ src["points"][i] + P[:, 3]
            e = mp["points"][j] - x
            M = np.linalg.inv(mp["cov"][j] + R0 @ src["cov"][i] @ R0.T)
            c += e @ M @ e
        return c

    assert abs(cost_at(pose, idx, np.zeros(6)) - cost) < 1e-9 * max(1.0, cost)
    h = 1e-6
    for k in range(6):
        d = np.zeros(6)
        d[k] = h
        fd = (cost_at(pose, idx, d) - cost_at(pose, idx, -d)) / (2 * h)
        assert abs(fd - 2 * g[k]) <= 1e-5 * max(1.0, abs(fd)), (k, fd, 2 * g[k])
    # at the true pose the residuals vanish (up to FP32 rounding of the map), so the
    # cost's second differences are the Gauss-Newton Hessian 2 J^T M J itself
    idx0 = G.correspond(src["points"], W.astype(np.float32), mp["points"], mp["normal"], 0.05)
    H0, g0, cost0, _ = G.gn_system(src["points"], src["cov"], mp["points"], mp["cov"], idx0, W)
    for k in range(6):
        for l in range(6):
            d1, d2 = np.zeros(6), np.zeros(6)
            d1[k] += 1e-4
            d2[l] += 1e-4
            sd = (cost_at(W, idx0, d1 + d2) - cost_at(W, idx0, d1 - d2) - cost_at(W, idx0, d2 - d1)
                  + cost_at(W, idx0, -d1 - d2)) / (4e-8)
            assert abs(sd - 2 * H0[k, l]) <= 1e-3 * abs(2 * H0).max(), (k, l, sd, 2 * H0[k, l])


def test_gicp_recovers_a_rigid_motion():
    rng = np.random.default_rng(5)
    src = _pair(rng)
    ang = math.radians(1.0)
    axis = np.array([0.2, 1.0, -0.3])
    W = np.hstack([G.exp_so3(ang * axis / np.linalg.norm(axis)), [[0.015], [-0.01], [0.012]]])
    mp = dict(points=G.transform32(W.astype(np.float32), src["points"]),
              cov=np.einsum("ij,mjk,lk->mil", W[:, :3], src["cov"], W[:, :3]),
              normal=src["normal"] @ W[:, :3].T)
    pose0 = np.hstack([np.eye(3), np.zeros((3, 1))])
    hist = []
    pose = G.gicp(src, mp, pose0, r_max=0.1, max_iters=30, tol=1e-7, history=hist)
    R_err = np.degrees(np.arccos(np.clip((np.trace(pose[:, :3] @ W[:, :3].T) - 1) / 2, -1, 1)))
    assert R_err < 0.01 and np.linalg.norm(pose[:, 3] - W[:, 3]) < 2e-4, (R_err, pose[:, 3] - W[:, 3])
    assert hist[-1]["cost"] < 1e-2 * hist[0]["cost"]


def test_insert_keeps_non_overlapping():
    src = dict(points=np.array([[0, 0, 1], [0.5, 0, 1], [0.011, 0, 1]], np.float32),
               cov=np.tile(np.eye(3), (3, 1, 1)), normal=np.tile([0.0, 0.0, 1.0], (3, 1)))
    mp = dict(points=np.array([[0.0, 0.0, 1.005]], np.float32), cov=np.eye(3)[None], normal=np.array([[0, 0, 1.0]]))
    pose = np.hstack([np.eye(3), np.zeros((3, 1))])
    out = G.insert(mp, src, pose, d_ov=0.01)
    assert list(out["added"]) == [1, 2]                     # point 0 is 5 mm from the map point
    assert len(out["points"]) == 3
    out2 = G.insert(G.empty_map(), src, pose, d_ov=0.01)
    assert list(out2["added"]) == [0, 1, 2]
