"""Pins of the oracle's single-precision decision path against the FP64 definition.

The oracle takes every discrete decision (near-plane cull, the integer radius, the tile
rectangle, power > 0, the alpha floor and cap, the transmittance stop) in FP32, the
precision the kernels take them in, so that keys, tile lists and contributor counts can
be compared bit for bit. Nothing else checks that FP32 path against the definition
(Sec. 3.2 and the 3DGS conventions of the projection and compositing; a1-a7 of the
path), so a slip copied into both the oracle and the kernels (a transposed index, a
wrong sign) would pass every parity test. Here the FP32 values the oracle decides with
(pixel mean, conic, opacity) are held to their FP64 counterparts within a rounding-error
bound derived from the FP32 operation sequence, and every FP32 decision must equal the
decision the FP64 values take, except where the threshold lies between the FP64 value
and the value the (pinned) FP32 inputs give, widened by the rounding of the last few
FP32 operations; those exceptions are counted and printed.

Error bound (eps = 2^-24, unit roundoff of FP32): with S_i = sum_j |V_ij| Smu_j + |V_i3|
the magnitude sum of the view-space coordinate t_i (Smu_j the same for the world
coordinate mu_j from the keyframe ray), each FP32 t_i carries at most 10 eps S_i (7
roundings in mu, 3 in t); the pixel mean p = f t_xy / t_z + c then carries at most
fx (dt_x + |u_x| dt_z) / t_z + 2 eps fx |u_x| + eps |p|, doubled for safety. The 2D
covariance is built from J = f / t_z terms, so the conic and the radius inherit twice the
relative error of t_z plus a few roundings; alpha = o exp(power) inherits the error of
power through the mean (|d power / d p| dp) and the conic (|power| times its relative
error); the transmittance stop inherits the accumulated relative errors of the alphas.
"""
import numpy as np
import pytest

import oracle
from paper_2603_21055_gb300 import synth

EPS = 2.0 ** -24


def _pixel_coords(kf):
    w, h = kf.cam.width, kf.cam.height
    j = np.arange(w * h)
    return (j % w).astype(np.float64), (j // w).astype(np.float64)


def error_bounds(scene, view_idx, P):
    """Per Gaussian: (bound on |pf - p| in x and y, relative error bound of t, of the
    conic), from the FP32 operation sequence (module docstring)."""
    v = scene.views[view_idx]
    V = np.asarray(v.pose, np.float64).reshape(3, 4)
    S_list = []
    for kf in scene.keyframes:
        M = np.asarray(kf.cam.pose, np.float64).reshape(3, 4)
        u, vv = _pixel_coords(kf)
        d = np.abs(kf.depth.astype(np.float64).ravel() + kf.offset.astype(np.float64).ravel())
        qx = d * (u - kf.cam.cx) / kf.cam.fx
        qy = d * (vv - kf.cam.cy) / kf.cam.fy
        smu = np.abs(M[:, 0:1] * qx) + np.abs(M[:, 1:2] * qy) + np.abs(M[:, 2:3] * d) + np.abs(M[:, 3:4])
        S_list.append(np.abs(V[:, :3]) @ smu + np.abs(V[:, 3:4]))
    S = np.concatenate(S_list, axis=1)                       # (3, n)
    dt = 10.0 * EPS * S
    tz = P["t"][:, 2]
    with np.errstate(divide="ignore", invalid="ignore"):
        ux, uy = P["t"][:, 0] / tz, P["t"][:, 1] / tz
        dpx = 2.0 * (v.fx * (dt[0] + np.abs(ux) * dt[2]) / np.abs(tz) + 2 * EPS * v.fx * np.abs(ux) +
                     EPS * np.abs(P["p"][:, 0]))
        dpy = 2.0 * (v.fy * (dt[1] + np.abs(uy) * dt[2]) / np.abs(tz) + 2 * EPS * v.fy * np.abs(uy) +
                     EPS * np.abs(P["p"][:, 1]))
        rel_t = dt.max(axis=0) / np.abs(tz)
    rel_conic = 8.0 * rel_t + 64.0 * EPS
    return dpx, dpy, dt[2], rel_conic, rel_t


def fp64_binning(scene, view_idx, P, o, bounds):
    """Cull, radius and tile rectangle from the FP64 projection (definition a2), and a
    near flag where the FP64 value lies within the FP32 error bound of a threshold."""
    v = scene.views[view_idx]
    dpx, dpy, dtz, rel_conic, rel_t = bounds
    tz = P["t"][:, 2]
    x, y, w = P["cov"][:, 0], P["cov"][:, 1], P["cov"][:, 2]
    det = x * w - y * y
    mid = 0.5 * (x + w)
    lam = mid + np.sqrt(np.maximum(0.1, mid * mid - det))
    r3 = 3.0 * np.sqrt(lam)
    rho = np.ceil(r3)
    px, py = P["p"][:, 0], P["p"][:, 1]
    x0, x1, y0, y1 = np.floor(px - rho), np.floor(px + rho), np.floor(py - rho), np.floor(py + rho)
    vis = (tz > 0.2) & (det > 0.0)
    off = (x1 < 0) | (y1 < 0) | (x0 > v.width - 1) | (y0 > v.height - 1)
    ix0, iy0 = np.maximum(x0, 0), np.maximum(y0, 0)
    ix1, iy1 = np.minimum(x1, v.width - 1), np.minimum(y1, v.height - 1)
    tx0, tx1 = (ix0 // o.tile_w).astype(np.int64), (ix1 // o.tile_w).astype(np.int64)
    ty0, ty1 = (iy0 // o.tile_h).astype(np.int64), (iy1 // o.tile_h).astype(np.int64)
    ntiles = np.where(vis & ~off, (tx1 - tx0 + 1) * (ty1 - ty0 + 1), 0)

    def gap(a):
        return np.abs(a - np.round(a))

    def straddle(v64, v32, slack):
        """An integer lies between the FP64 and the FP32-input value (floor may differ)."""
        lo, hi = np.minimum(v64, v32) - slack, np.maximum(v64, v32) + slack
        return np.floor(lo) != np.floor(hi)

    near = np.abs(tz - 0.2) <= 2.0 * dtz
    live = vis & ~near
    # r3 = 3 sqrt(lambda): lambda carries twice the relative error of J (2 rel_t) plus
    # ~12 roundings, r3 half of that plus two: (rel_t + 8 eps), doubled
    near_r = live & (gap(r3) <= r3 * (2.0 * rel_t + 16.0 * EPS))
    # the rectangle is floor(pf -+ rho) of the FP32 mean: ambiguous only where an integer
    # lies between p -+ rho and pf -+ rho (+- the rounding of that subtraction)
    pfx, pfy = P["pf"][:, 0].astype(np.float64), P["pf"][:, 1].astype(np.float64)
    sx, sy = 2 * EPS * (np.abs(px) + rho), 2 * EPS * (np.abs(py) + rho)
    near_p = live & (straddle(px - rho, pfx - rho, sx) | straddle(px + rho, pfx + rho, sx) |
                     straddle(py - rho, pfy - rho, sy) | straddle(py + rho, pfy + rho, sy))
    near = near | near_r | near_p
    return dict(visible=vis, rho=rho, tx0=tx0, tx1=tx1, ty0=ty0, ty1=ty1, ntiles=ntiles, near=near)


def check_projection(scene, o):
    """Every view: FP32 values within their bounds, FP32 decisions equal to FP64 ones
    away from thresholds. Returns (Gaussians checked, near exceptions, exceptions whose
    FP32 decisions nevertheless equal the FP64 ones)."""
    n_checked, n_near, n_near_agree = 0, 0, 0
    for k in range(len(scene.views)):
        P = oracle.project(scene, k, o)
        b = error_bounds(scene, k, P)
        dpx, dpy, dtz, rel_conic, _ = b
        d = fp64_binning(scene, k, P, o, b)
        vis = P["visible"] != 0
        # values the decisions are taken with
        assert np.all(np.abs(P["pf"][vis, 0] - P["p"][vis, 0]) <= dpx[vis])
        assert np.all(np.abs(P["pf"][vis, 1] - P["p"][vis, 1]) <= dpy[vis])
        scale = np.maximum(np.abs(P["conic"][:, 0]), np.abs(P["conic"][:, 2]))
        err_c = np.abs(P["conicf"].astype(np.float64) - P["conic"]).max(axis=1)
        assert np.all(err_c[vis] <= rel_conic[vis] * scale[vis]), float((err_c / (rel_conic * scale))[vis].max())
        assert np.all(np.abs(P["of"] - P["o"]) <= 4.0 * EPS * P["o"])
        # decisions
        keep = ~d["near"]
        np.testing.assert_array_equal(vis[keep], d["visible"][keep])
        both = keep & vis
        np.testing.assert_array_equal(P["rho"][both], d["rho"][both])
        np.testing.assert_array_equal(P["ntiles"][keep], d["ntiles"][keep])
        has = both & (d["ntiles"] > 0)
        for q in ("tx0", "tx1", "ty0", "ty1"):
            np.testing.assert_array_equal(P[q][has], d[q][has])
        n_checked += int(keep.sum())
        n_near += int(d["near"].sum())
        agree = d["near"] & (vis == d["visible"]) & (P["ntiles"] == d["ntiles"])
        agree &= ~vis | (P["rho"] == d["rho"])
        for q in ("tx0", "tx1", "ty0", "ty1"):
            agree &= (d["ntiles"] == 0) | (P[q] == d[q])
        n_near_agree += int(agree.sum())
    return n_checked, n_near, n_near_agree


def fp64_walk(P, list_g, qx, qy):
    """Front-to-back walk (definition a7) of one pixel over a tile list, every decision
    in FP64, with a near flag where a threshold lies between the FP64 decision value and
    the one the oracle's FP32 inputs (pf, conicf, of; pinned to the FP64 ones by
    check_projection) give, widened by the rounding of the FP32 power expression (6 eps
    of its terms), of expf and the opacity product (4 eps) and, for the stop, of the
    running FP32 product (2 eps per factor). Returns (rgb, depth, alpha, T, index of the
    last contributor in list_g or -1, near)."""
    g = list_g

    def alpha_of(p, conic, o):
        dx, dy = p[g, 0] - qx, p[g, 1] - qy
        a, b, c = conic[g, 0], conic[g, 1], conic[g, 2]
        power = -0.5 * (a * dx * dx + c * dy * dy) - b * dx * dy
        mag = 0.5 * (np.abs(a) * dx * dx + np.abs(c) * dy * dy) + np.abs(b * dx * dy)
        return power, o[g] * np.exp(power), mag

    power, raw, _ = alpha_of(P["p"], P["conic"], P["o"])
    pw32, raw32, mag = alpha_of(P["pf"].astype(np.float64), P["conicf"].astype(np.float64),
                                P["of"].astype(np.float64))
    sp = 6.0 * EPS * mag                                        # power rounding
    sr = (sp + 4.0 * EPS) * raw32                               # alpha rounding

    def straddles(x64, x32, slack, thr):
        return (np.minimum(x64, x32 - slack) <= thr) & (np.maximum(x64, x32 + slack) >= thr)

    near_e = (straddles(power, pw32, sp, 0.0) | straddles(raw, raw32, sr, 0.99) |
              straddles(raw, raw32, sr, 1.0 / 255.0))
    alpha = np.minimum(0.99, raw)
    alpha32 = np.minimum(0.99, raw32)
    take = (power <= 0.0) & (alpha >= 1.0 / 255.0)
    T, T32, rel32 = 1.0, 1.0, 0.0
    rgb, depth, acc = np.zeros(3), 0.0, 0.0
    last, near = -1, False
    for i in np.nonzero(take | near_e)[0]:
        near |= bool(near_e[i])
        if not take[i]:
            continue
        test = T * (1.0 - alpha[i])
        test32 = T32 * (1.0 - alpha32[i])
        rel = rel32 + (alpha32[i] / (1.0 - alpha32[i])) * (sr[i] / raw32[i]) * (raw32[i] <= 0.99) + 2.0 * EPS
        if straddles(test, test32, rel * test32, 1e-4):
            near = True
        if test < 1e-4:
            break
        w = alpha[i] * T
        rgb += w * P["color"][g[i]]
        depth += w * P["t"][g[i], 2]
        acc += w
        T, T32, rel32, last = test, test32, rel, i
    return rgb, depth, acc, T, last, near


def check_walks(scene, o, n_tiles=None, px_per_tile=None, seed=0):
    """Sampled (or all) pixels of every view: the oracle's FP32-decided walk against the
    FP64 one. A pixel is set aside (counted) when a decision of either walk is near, when
    a Gaussian that reaches it (FP64 alpha >= 1/510) is listed in its tile by one
    rectangle and not the other, or when the f32 rounding of a listed depth is near."""
    rng = np.random.default_rng(seed)
    n_checked, n_near = 0, 0
    for k, v in enumerate(scene.views):
        P = oracle.project(scene, k, o)
        b = error_bounds(scene, k, P)
        d = fp64_binning(scene, k, P, o, b)
        ntx, nty = (v.width + o.tile_w - 1) // o.tile_w, (v.height + o.tile_h - 1) // o.tile_h
        tiles = np.arange(ntx * nty) if n_tiles is None else rng.choice(ntx * nty, min(n_tiles, ntx * nty), False)
        zb = P["zf"].astype(np.float32)
        work = []
        for t in tiles:
            tx, ty = t % ntx, t // ntx
            cov64 = (d["ntiles"] > 0) & (d["tx0"] <= tx) & (d["tx1"] >= tx) & (d["ty0"] <= ty) & (d["ty1"] >= ty)
            cov32 = (P["ntiles"] > 0) & (P["tx0"] <= tx) & (P["tx1"] >= tx) & (P["ty0"] <= ty) & (P["ty1"] >= ty)
            differ = np.nonzero(cov64 != cov32)[0]
            z_near = bool(((P["near"] != 0) & cov32).any())
            g = np.nonzero(cov64)[0]
            g = g[np.lexsort((g, zb[g]))]
            # n_contrib is a position in the list the FP32 rectangles define (pinned by
            # check_projection); the walk itself runs over the FP64 list
            g32 = np.nonzero(cov32)[0]
            g32 = g32[np.lexsort((g32, zb[g32]))]
            pos32 = {int(x): i for i, x in enumerate(g32)}
            xs = np.arange(tx * o.tile_w, min((tx + 1) * o.tile_w, v.width))
            ys = np.arange(ty * o.tile_h, min((ty + 1) * o.tile_h, v.height))
            X, Y = np.meshgrid(xs, ys)
            X, Y = X.ravel(), Y.ravel()
            if px_per_tile is not None and len(X) > px_per_tile:
                s = rng.choice(len(X), px_per_tile, replace=False)
                X, Y = X[s], Y[s]
            work.append((g, pos32, differ, z_near, X, Y))
        allx = np.concatenate([w[4] for w in work])
        ally = np.concatenate([w[5] for w in work])
        ref = oracle.render_pixels(scene, np.full(len(allx), k), allx, ally, o)
        i0 = 0
        for g, pos32, differ, z_near, X, Y in work:
            for i in range(len(X)):
                r = i0 + i
                qx, qy = float(X[i]), float(Y[i])
                rgb, depth, acc, T, last, near = fp64_walk(P, g, qx, qy)
                if len(differ):
                    dx, dy = P["p"][differ, 0] - qx, P["p"][differ, 1] - qy
                    cn = P["conic"][differ]
                    pw = -0.5 * (cn[:, 0] * dx * dx + cn[:, 2] * dy * dy) - cn[:, 1] * dx * dy
                    near |= bool((P["o"][differ] * np.exp(np.minimum(pw, 0.0)) >= 0.5 / 255.0).any())
                if near or z_near or ref["near"][r] or (last >= 0 and int(g[last]) not in pos32):
                    n_near += 1
                    continue
                nc = pos32[int(g[last])] + 1 if last >= 0 else 0
                assert ref["n_contrib"][r] == nc, (k, qx, qy, ref["n_contrib"][r], nc)
                np.testing.assert_allclose(ref["rgb"][r], rgb, rtol=0, atol=1e-12)
                assert abs(ref["depth"][r] - depth) <= 1e-12 and abs(ref["alpha"][r] - acc) <= 1e-12
                assert abs(ref["t_final"][r] - T) <= 1e-12
                n_checked += 1
            i0 += len(X)
    return n_checked, n_near


def test_projection_decisions_plane(scene1):
    """The 64x48 plane: FP32 values within bound, decisions equal, no exception."""
    n, near, agree = check_projection(scene1, oracle.opts())
    print("plane: %d Gaussians' binning decisions equal to FP64, %d near a threshold (%d of them equal)" %
          (n, near, agree))
    assert near == 0 and n == scene1.n_gaussians


def test_projection_decisions_room_views():
    """All 2.46M Gaussians of the 8-keyframe room in each of its 8 views (16x16 tiles)
    and in one view with 8x32 tiles."""
    room = synth.config2_room()
    n, near, agree = check_projection(room, oracle.opts())
    print("room: %d (Gaussian, view) binning decisions equal to FP64, %d near a threshold (%d of them equal)" %
          (n, near, agree))
    # ~2.3e-4 of the pairs: a rectangle edge with an integer between the FP64 and the
    # FP32 mean, or 3 sqrt(lambda) within its error bound of an integer
    assert near <= 5e-4 * n
    one = synth.Scene(room.keyframes, room.views[:1], room.target_rgb[:1], room.target_depth[:1])
    n2, near2, _ = check_projection(one, oracle.opts(tile_w=8, tile_h=32))
    assert near2 <= 5e-4 * n2


def test_walk_decisions_plane(scene1):
    """Every pixel of the plane: the oracle's FP32-decided walk (accepted entries,
    stop, contributor count) equals the FP64-decided walk of the definition."""
    n, near = check_walks(scene1, oracle.opts())
    print("plane walks: %d pixels equal to the FP64 walk, %d near a threshold" % (n, near))
    assert n + near == 64 * 48 and near <= 0.01 * (n + near)


def test_walk_decisions_room_crop(room2):
    """Every pixel of the two-view room crop (3 keyframes, 120x90 views) and sampled
    pixels of 16 full-size room tiles (8 in each of two views)."""
    crop = synth.crop_scene(room2, (260, 200, 100, 70), (250, 190, 120, 90), n_keyframes=3, n_views=2)
    n, near = check_walks(crop, oracle.opts())
    print("crop walks: %d pixels equal to the FP64 walk, %d near a threshold" % (n, near))
    # FP32 means carry up to ~3e-4 px of rounding error, i.e. ~7e-4 relative in alpha at
    # the floor's ellipse: a pixel that evaluates a few hundred entries meets one whose
    # FP64 and FP32 alphas straddle 1/255 about once in twenty (4.9 % measured)
    assert near <= 0.08 * (n + near)
    one = synth.Scene(room2.keyframes, room2.views[:2], room2.target_rgb[:2], room2.target_depth[:2])
    n2, near2 = check_walks(one, oracle.opts(), n_tiles=8, px_per_tile=12, seed=3)
    print("room walks: %d pixels equal to the FP64 walk, %d near a threshold" % (n2, near2))
    # full-size tiles: a pixel walks ~1,200 entries before its stop, four times the
    # crop's, so a straddled alpha floor is four times as likely (~10 % measured)
    assert near2 <= 0.2 * (n2 + near2)


@pytest.mark.parametrize("tile", [(16, 16), (32, 8)])
def test_other_tile_shapes(scene1, tile):
    o = oracle.opts(tile_w=tile[0], tile_h=tile[1])
    n, near, _ = check_projection(scene1, o)
    assert near == 0
    n, near = check_walks(scene1, o, n_tiles=4)
    assert near <= 0.01 * (n + near)
