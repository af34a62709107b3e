"""Oracle of the geometric tracking (Sec. 3.3 "Matching a Frame to a Scene", "Generalized
ICP for Matching", Eq. 2; scale normalisation of the ablations; R and K_c of Supp. A).

TEST INFRASTRUCTURE ONLY: the tests and the CPU leg of the benchmark may call it; the
CUDA path never does, and it shares no code with the library. Plain numpy, FP64, except
where floating point decides an integer (which points are neighbours, which map
Gaussian a source Gaussian corresponds to, which source Gaussians overlap the map):
those decisions are taken in FP32 with the same operation order as the library, as
stated at each function. scipy's KD-tree, where used, only pre-selects candidates with a
padded radius; the decision itself is the FP32 test.

Readings (the paper is silent or garbled):
  * Selection: the pixels (u, v) with u and v multiples of R and depth > 0, in raster
    order, back-projected to p = d ((u - cx) / fx, (v - cy) / fy, 1).
  * Neighbours: the K_c nearest selected points of the same frame, the point itself
    included, by FP32 squared distance ((dx dx + dy dy) + dz dz), ties by index (all of
    them when the frame has fewer than K_c points).
  * Covariance: (1 / K_c) sum (p - m)(p - m)^T over those points; its eigen-decomposition
    (the SVD of a symmetric PSD matrix) gives scales s_k = sqrt(lambda_k) and rotation.
  * Scale normalisation: s <- s / max(s), each normalised scale floored at sqrt(1e-3)
    (Segal et al.'s epsilon, so the matrix stays invertible); C = V diag(s^2) V^T; the
    normal is the eigenvector of the smallest scale. A degenerate set (all points equal)
    gets s = (1, 1, 1).
  * Correspondence: for the source point moved into the world, x = R a + t (FP32), the
    candidates are its k_match = 5 nearest map Gaussians b within r_max (FP32 squared
    distance <= r_max^2, ties by index), and the one with the smallest point-to-surface
    distance |n_b . (mu_b - x)| wins, ties by squared distance, then index; none in range
    -> no correspondence. (Taking the surface distance over every Gaussian within r_max
    leaves the position along the surface unconstrained; over the nearest few it keeps
    the robustness to depth noise the paper reports against point-to-point matching:
    with 2 mm noise on resampled surfaces, 5 candidates gave about a third of the
    translation error of the Euclidean nearest one.)
  * Eq. 2 is printed without the inverse; it is read as the GICP objective of Segal et
    al.: sum e^T (C_b + R C_a R^T)^-1 e, e = mu_b - (R a + t), minimised by Gauss-Newton
    on a left perturbation x -> x + omega x x + v (Jacobian [[x]_x, -I], the covariance
    term held fixed within an iteration), step xi = -H^-1 g, update
    (R, t) <- (Exp(omega) R, Exp(omega) t + v); stop when |xi| < tol or after max_iters.
  * Map update: a source Gaussian joins the map unless a map Gaussian lies within d_ov
    of it (FP32 squared distance <= d_ov^2), in source order; its covariance is rotated
    into the world (R C R^T) and its normal with it.
"""
from __future__ import annotations

import math

import numpy as np

EPS = 1e-3
F32 = np.float32


# --------------------------------------------------------------------------- selection
def select_points(depth: np.ndarray, fx: float, fy: float, cx: float, cy: float, R: int):
    """Selected points (M, 3) float32 in the camera frame and their pixel indices."""
    depth = np.asarray(depth, F32)
    h, w = depth.shape
    vs, us = np.meshgrid(np.arange(0, h, R), np.arange(0, w, R), indexing="ij")
    vs, us = vs.ravel(), us.ravel()
    d = depth[vs, us]
    keep = d > 0
    vs, us, d = vs[keep], us[keep], d[keep]
    fx, fy, cx, cy = F32(fx), F32(fy), F32(cx), F32(cy)
    x = d * ((us.astype(F32) - cx) / fx)
    y = d * ((vs.astype(F32) - cy) / fy)
    pts = np.stack([x, y, d], 1).astype(F32)
    return pts, vs * w + us


# --------------------------------------------------------------------------- neighbours
def sqdist32(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """FP32 squared distances ((dx dx + dy dy) + dz dz) between rows of a (n,3) and b (m,3)."""
    a, b = np.asarray(a, F32), np.asarray(b, F32)
    dx = b[None, :, 0] - a[:, None, 0]
    dy = b[None, :, 1] - a[:, None, 1]
    dz = b[None, :, 2] - a[:, None, 2]
    return (dx * dx + dy * dy) + dz * dz


def knn(points: np.ndarray, K: int, chunk: int = 512) -> np.ndarray:
    """(M, min(K, M)) indices of each point's K nearest points (itself included), FP32
    distances, ties by index (all M points when there are fewer than K)."""
    P = np.asarray(points, F32)
    K = min(K, len(P))
    out = np.empty((len(P), K), np.int64)
    for s in range(0, len(P), chunk):
        D = sqdist32(P[s:s + chunk], P)
        out[s:s + chunk] = np.argsort(D, axis=1, kind="stable")[:, :K]
    return out


# --------------------------------------------------------------------------- shapes
def covariances(points: np.ndarray, idx: np.ndarray) -> np.ndarray:
    Q = np.asarray(points, np.float64)[idx]                  # (M, K, 3)
    d = Q - Q.mean(axis=1, keepdims=True)
    return np.einsum("mki,mkj->mij", d, d) / idx.shape[1]


def normalised_shapes(cov: np.ndarray):
    """(normalised covariances (M,3,3), normals (M,3), raw scales (M,3) ascending)."""
    w, V = np.linalg.eigh(cov)                               # ascending eigenvalues
    s = np.sqrt(np.maximum(w, 0.0))
    smax = s[:, 2:3]
    sn = np.where(smax > 0, s / np.where(smax > 0, smax, 1.0), 1.0)
    sn = np.maximum(sn, math.sqrt(EPS))
    Cn = np.einsum("mij,mj,mkj->mik", V, sn * sn, V)
    return Cn, V[:, :, 0], s


def frame_gaussians(depth, fx, fy, cx, cy, R: int, K: int):
    """T_i of a depth map: points (camera frame, float32), normalised covariances,
    normals, K-neighbour indices."""
    pts, pix = select_points(depth, fx, fy, cx, cy, R)
    idx = knn(pts, K)
    C, n, s = normalised_shapes(covariances(pts, idx))
    return dict(points=pts, cov=C, normal=n, pix=pix, knn=idx, scales=s)


# --------------------------------------------------------------------------- matching
def transform32(pose: np.ndarray, a: np.ndarray) -> np.ndarray:
    """x = R a + t in FP32, each row as ((r0 a0 + r1 a1) + r2 a2) + t."""
    P = np.asarray(pose, F32)
    a = np.asarray(a, F32)
    cols = []
    for r in range(3):
        cols.append(((P[r, 0] * a[:, 0] + P[r, 1] * a[:, 1]) + P[r, 2] * a[:, 2]) + P[r, 3])
    return np.stack(cols, 1).astype(F32)


K_MATCH = 5


def correspond(src_points, pose, map_points, map_normals, r_max: float, k_match: int = K_MATCH) -> np.ndarray:
    """Index of each source point's map Gaussian (or -1): among its k_match nearest map
    points within r_max (FP32, ties by index), the smallest FP32 point-to-surface
    distance, ties by squared distance, then index."""
    from scipy.spatial import cKDTree
    x = transform32(pose, src_points)
    B = np.asarray(map_points, F32)
    N = np.asarray(map_normals, F32)
    r2 = F32(r_max) * F32(r_max)
    tree = cKDTree(B.astype(np.float64))
    cand = tree.query_ball_point(x.astype(np.float64), r=float(r_max) * (1 + 1e-4) + 1e-7)
    out = np.full(len(x), -1, np.int64)
    for i, c in enumerate(cand):
        if not c:
            continue
        c = np.asarray(sorted(c), np.int64)
        dx = B[c, 0] - x[i, 0]
        dy = B[c, 1] - x[i, 1]
        dz = B[c, 2] - x[i, 2]
        d2 = (dx * dx + dy * dy) + dz * dz
        ok = d2 <= r2
        if not ok.any():
            continue
        c, dx, dy, dz, d2 = c[ok], dx[ok], dy[ok], dz[ok], d2[ok]
        near = np.lexsort((c, d2))[:k_match]                  # nearest first, ties by index
        c, dx, dy, dz, d2 = c[near], dx[near], dy[near], dz[near], d2[near]
        m = np.abs((N[c, 0] * dx + N[c, 1] * dy) + N[c, 2] * dz)
        order = np.lexsort((c, d2, m))                       # by m, then d2, then index
        out[i] = c[order[0]]
    return out


def skew(v):
    return np.array([[0, -v[2], v[1]], [v[2], 0, -v[0]], [-v[1], v[0], 0]])


def gn_system(src_points, src_cov, map_points, map_cov, idx, pose):
    """(H (6,6), g (6,), cost, n) of Eq. 2 at `pose` (FP64) for the given correspondences."""
    P = np.asarray(pose, np.float64)
    R, t = P[:, :3], P[:, 3]
    H = np.zeros((6, 6))
    g = np.zeros(6)
    cost, n = 0.0, 0
    for i, j in enumerate(idx):
        if j < 0:
            continue
        a = np.asarray(src_points[i], np.float64)
        x = R @ a + t
        e = np.asarray(map_points[j], np.float64) - x
        M = np.linalg.inv(np.asarray(map_cov[j], np.float64) + R @ np.asarray(src_cov[i], np.float64) @ R.T)
        J = np.hstack([skew(x), -np.eye(3)])
        H += J.T @ M @ J
        g += J.T @ M @ e
        cost += e @ M @ e
        n += 1
    return H, g, cost, n


def exp_so3(w):
    th = float(np.linalg.norm(w))
    K = skew(w)
    if th < 1e-12:
        return np.eye(3) + K
    return np.eye(3) + math.sin(th) / th * K + (1 - math.cos(th)) / th ** 2 * (K @ K)


def apply_step(pose, xi):
    """(R, t) <- (Exp(omega) R, Exp(omega) t + v)."""
    P = np.asarray(pose, np.float64)
    E = exp_so3(np.asarray(xi[:3], np.float64))
    return np.hstack([E @ P[:, :3], (E @ P[:, 3] + np.asarray(xi[3:], np.float64))[:, None]])


def gicp(src, map_, pose0, r_max: float, max_iters: int = 30, tol: float = 1e-6, history=None,
         k_match: int = K_MATCH):
    """Camera pose (cam -> world 3x4, FP64) of the source Gaussians against the map."""
    pose = np.asarray(pose0, np.float64)
    for it in range(max_iters):
        idx = correspond(src["points"], pose.astype(F32), map_["points"], map_["normal"], r_max, k_match)
        H, g, cost, n = gn_system(src["points"], src["cov"], map_["points"], map_["cov"], idx, pose)
        if n < 6:
            break
        xi = -np.linalg.solve(H, g)
        pose = apply_step(pose, xi)
        if history is not None:
            history.append(dict(cost=cost, n=n, step=float(np.linalg.norm(xi))))
        if np.linalg.norm(xi) < tol:
            break
    return pose


def insert(map_, src, pose, d_ov: float):
    """The map after adding the source Gaussians no map Gaussian overlaps (world frame)."""
    from scipy.spatial import cKDTree
    x = transform32(np.asarray(pose, F32), src["points"])
    B = np.asarray(map_["points"], F32)
    keep = np.ones(len(x), bool)
    if len(B):
        tree = cKDTree(B.astype(np.float64))
        cand = tree.query_ball_point(x.astype(np.float64), r=float(d_ov) * (1 + 1e-4) + 1e-7)
        r2 = F32(d_ov) * F32(d_ov)
        for i, c in enumerate(cand):
            if c:
                c = np.asarray(c, np.int64)
                dx = B[c, 0] - x[i, 0]
                dy = B[c, 1] - x[i, 1]
                dz = B[c, 2] - x[i, 2]
                if (((dx * dx + dy * dy) + dz * dz) <= r2).any():
                    keep[i] = False
    R = np.asarray(pose, np.float64)[:, :3]
    cov_w = np.einsum("ij,mjk,lk->mil", R, src["cov"][keep], R)
    n_w = src["normal"][keep] @ R.T
    return dict(points=np.concatenate([B, x[keep]]).astype(F32),
                cov=np.concatenate([np.asarray(map_["cov"]).reshape(-1, 3, 3), cov_w]),
                normal=np.concatenate([np.asarray(map_["normal"], np.float64).reshape(-1, 3), n_w]),
                added=np.nonzero(keep)[0])


def empty_map():
    return dict(points=np.zeros((0, 3), F32), cov=np.zeros((0, 3, 3)), normal=np.zeros((0, 3)))
