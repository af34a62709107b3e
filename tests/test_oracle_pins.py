"""Pins of the FP64 oracle against facts that do not come from the oracle itself:
closed forms, geometric identities, brute force on tiny inputs and finite differences.

Each test names the passage or property it rests on. A plausible slip in the oracle (a
dropped term, a wrong sign or index, a transposed pose, a wrong bound) fails one of them.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2603_21055_gb300.synth import Camera, Keyframe, Scene, pose_inverse, rotation_about

ALPHA_FLOOR = 1.0 / 255.0


def sigmoid(x):
    return 1.0 / (1.0 + math.exp(-x))


def one_gaussian_kf(depth, logit, color, scale, f=64.0, pose=None):
    """A 1x1 keyframe whose single pixel ray is the optical axis (cx = cy = 0)."""
    pose = np.concatenate([np.eye(3), np.zeros((3, 1))], 1) if pose is None else pose
    cam = Camera(1, 1, f, f, 0.0, 0.0, np.asarray(pose, np.float32))
    a = lambda v: np.full((1, 1), v, np.float32)
    return Keyframe(cam, a(depth), a(0.0), np.asarray(color, np.float32).reshape(3, 1, 1), a(logit), a(scale))


def identity_view(w=32, h=32, f=64.0, cx=16.0, cy=16.0):
    return Camera(w, h, f, f, cx, cy, np.concatenate([np.eye(3), np.zeros((3, 1))], 1).astype(np.float32))


def scene_of(kfs, views):
    return Scene(kfs, views, [np.zeros((3, v.height, v.width), np.float32) for v in views],
                 [np.zeros((v.height, v.width), np.float32) for v in views])


def random_scene(seed, n_kf=2, kw=12, kh=10, views=((20, 18),), f=18.0, logit_mean=1.0):
    rng = np.random.default_rng(seed)
    kfs = []
    for _ in range(n_kf):
        c2w = np.concatenate([rotation_about(rng.normal(size=3), math.radians(3.0)),
                              rng.normal(0, 0.03, size=(3, 1))], 1)
        cam = Camera(kw, kh, f, f, kw / 2.0, kh / 2.0, c2w.astype(np.float32))
        depth = rng.uniform(1.0, 2.0, size=(kh, kw)).astype(np.float32)
        kfs.append(Keyframe(cam, depth, rng.normal(0, 0.05, (kh, kw)).astype(np.float32),
                            rng.uniform(0, 1, (3, kh, kw)).astype(np.float32),
                            rng.normal(logit_mean, 0.7, (kh, kw)).astype(np.float32),
                            (depth / f * rng.uniform(0.8, 1.6, (kh, kw))).astype(np.float32)))
    vs = []
    for (w, h) in views:
        c2w = np.concatenate([rotation_about(rng.normal(size=3), math.radians(2.0)),
                              rng.normal(0, 0.03, size=(3, 1))], 1)
        vs.append(Camera(w, h, f * 1.3, f * 1.3, w / 2.0, h / 2.0, pose_inverse(c2w).astype(np.float32)))
    return scene_of(kfs, vs)


# ------------------------------------------------------------------ geometry pins

def test_self_projection_identity_exact_pose():
    """Sec. 3.2: Gaussian j sits on the ray of pixel j at depth |D + delta|, so in its own
    keyframe's view it projects exactly onto the pixel centre with t_z = |D + delta|.
    The pose is an exact axis permutation with a dyadic translation, so every float32
    input is exact and the identity holds to FP64 rounding."""
    rng = np.random.default_rng(0)
    perm = np.array([[0, 0, 1], [1, 0, 0], [0, 1, 0]], np.float64)
    c2w = np.concatenate([perm, np.array([[0.5], [-1.25], [2.0]])], 1)
    W, H, f = 24, 20, 30.0
    depth = rng.uniform(0.5, 4.0, (H, W)).astype(np.float32)
    offset = rng.normal(0.0, 0.3, (H, W)).astype(np.float32)
    offset[0, 0] = -2.0 * depth[0, 0] - 0.5        # D + delta < 0: placed at |D + delta|
    cam = Camera(W, H, f, f, 11.5, 9.5, c2w.astype(np.float32))
    kf = Keyframe(cam, depth, offset, rng.uniform(0, 1, (3, H, W)).astype(np.float32),
                  np.zeros((H, W), np.float32), (depth / f).astype(np.float32))
    view = Camera(W, H, f, f, 11.5, 9.5, pose_inverse(c2w).astype(np.float32))
    P = oracle.project(scene_of([kf], [view]), 0)
    u, v = np.meshgrid(np.arange(W), np.arange(H))
    np.testing.assert_allclose(P["p"][:, 0], u.ravel(), atol=1e-12)
    np.testing.assert_allclose(P["p"][:, 1], v.ravel(), atol=1e-12)
    adj = np.abs(depth.astype(np.float64) + offset.astype(np.float64)).ravel()
    np.testing.assert_allclose(P["t"][:, 2], adj, rtol=1e-14)


def test_self_projection_identity_random_pose(scene1):
    """Same identity through an arbitrary float32 pose and its float32 inverse: holds to
    the float32 rounding of the poses."""
    rng = np.random.default_rng(1)
    c2w = np.concatenate([rotation_about(rng.normal(size=3), 0.7), rng.normal(size=(3, 1))], 1)
    k = scene1.keyframes[0]
    cam = Camera(k.cam.width, k.cam.height, k.cam.fx, k.cam.fy, k.cam.cx, k.cam.cy, c2w.astype(np.float32))
    kf = Keyframe(cam, k.depth, np.zeros_like(k.offset), k.rgb, k.logit, k.scale)
    view = Camera(cam.width, cam.height, cam.fx, cam.fy, cam.cx, cam.cy,
                  pose_inverse(cam.pose.astype(np.float64)).astype(np.float32))
    P = oracle.project(scene_of([kf], [view]), 0)
    u, v = np.meshgrid(np.arange(cam.width), np.arange(cam.height))
    np.testing.assert_allclose(P["p"][:, 0], u.ravel(), atol=2e-4)
    np.testing.assert_allclose(P["p"][:, 1], v.ravel(), atol=2e-4)
    np.testing.assert_allclose(P["t"][:, 2], k.depth.ravel(), rtol=1e-5)


def test_sigma2d_closed_form_principal_point():
    """EWA with the 0.3 px dilation: a Gaussian on the optical axis at depth z with scale
    s = z/fx (the r = D/F initialisation, Supp. A) has Sigma_2D = diag(1.3, 1.3), conic
    diag(1/1.3) and square radius ceil(3 sqrt(1.3 + sqrt(0.1))) = 4."""
    kf = one_gaussian_kf(2.0, 0.0, (1, 1, 1), 2.0 / 64.0)
    P = oracle.project(scene_of([kf], [identity_view()]), 0)[0]
    np.testing.assert_allclose(P["cov"], [1.3, 0.0, 1.3], atol=1e-15)
    np.testing.assert_allclose(P["conic"], [1 / 1.3, 0.0, 1 / 1.3], rtol=1e-14)
    np.testing.assert_allclose(P["p"], [16.0, 16.0], atol=0)
    assert P["rho"] == 4.0 == math.ceil(3 * math.sqrt(1.3 + math.sqrt(0.1)))
    assert (P["tx0"], P["tx1"], P["ty0"], P["ty1"]) == (0, 1, 0, 1)


def test_covariance_jacobian_matches_projection_fd(scene1):
    """The J in Sigma_2D = s^2 J J^T + 0.3 I must be the derivative of the projected mean
    with respect to the view-space centre: move the view translation by +-h along each
    axis (t changes by exactly that) and difference the projected means."""
    base = scene1.views[0]
    rng = np.random.default_rng(3)
    idx = rng.choice(scene1.n_gaussians, 20, replace=False)
    P0 = oracle.project(scene1, 0)
    h = 1e-6
    J = np.zeros((len(idx), 2, 3))
    for a in range(3):
        ps = []
        for sgn in (1, -1):
            pose = base.pose.astype(np.float64).copy()
            pose[a, 3] += sgn * h
            v = Camera(base.width, base.height, base.fx, base.fy, base.cx, base.cy, pose)
            sc = Scene(scene1.keyframes, [v], scene1.target_rgb, scene1.target_depth)
            ps.append(oracle.project(sc, 0)["p"][idx])
        J[:, :, a] = (ps[0] - ps[1]) / (2 * h)
    s2 = P0["s"][idx] ** 2
    cov = s2[:, None, None] * np.einsum("nij,nkj->nik", J, J) + 0.3 * np.eye(2)
    np.testing.assert_allclose(P0["cov"][idx, 0], cov[:, 0, 0], rtol=1e-7)
    np.testing.assert_allclose(P0["cov"][idx, 1], cov[:, 0, 1], rtol=1e-6, atol=1e-9)
    np.testing.assert_allclose(P0["cov"][idx, 2], cov[:, 1, 1], rtol=1e-7)


def test_conic_is_inverse_covariance(scene1):
    P = oracle.project(scene1, 0)
    P = P[P["ntiles"] > 0]
    for r in P[:50]:
        S = np.array([[r["cov"][0], r["cov"][1]], [r["cov"][1], r["cov"][2]]])
        Q = np.array([[r["conic"][0], r["conic"][1]], [r["conic"][1], r["conic"][2]]])
        np.testing.assert_allclose(S @ Q, np.eye(2), atol=1e-13)
        lam = np.linalg.eigvalsh(S).max()
        assert r["rho"] >= 3 * math.sqrt(lam)          # the bound covers 3 sigma


# ------------------------------------------------------------ compositing pins

@pytest.mark.parametrize("logit", [1.3, 9.0])
def test_single_gaussian_closed_form(logit):
    """One Gaussian seen from its own pose with Sigma_2D = 1.3 I: alpha(pixel) =
    min(0.99, sigmoid(logit) exp(-|pixel - p|^2 / 2.6)) where it is >= 1/255, else 0;
    RGB = alpha c, D = alpha z, A = alpha (black background). logit = 9 exercises the cap."""
    c = (0.2, 0.5, 0.9)
    kf = one_gaussian_kf(2.0, logit, c, 2.0 / 64.0)
    out = oracle.render(scene_of([kf], [identity_view()]))[0]
    y, x = np.mgrid[0:32, 0:32]
    a = np.minimum(0.99, sigmoid(logit) * np.exp(-((x - 16.0) ** 2 + (y - 16.0) ** 2) / 2.6))
    a = np.where(a >= ALPHA_FLOOR, a, 0.0)
    for ch in range(3):
        np.testing.assert_allclose(out["rgb"][ch], a * c[ch], atol=1e-12)
    np.testing.assert_allclose(out["depth"], a * 2.0, atol=1e-12)
    np.testing.assert_allclose(out["alpha"], a, atol=1e-12)
    np.testing.assert_allclose(out["t_final"], 1.0 - a, atol=1e-12)
    np.testing.assert_array_equal(out["n_contrib"], (a > 0).astype(np.int32))


@pytest.mark.parametrize("swap", [False, True])
def test_two_gaussians_ordering_closed_form(swap):
    """Front-to-back compositing of two Gaussians on the same ray: C = a1 c1 + (1 - a1)
    a2 c2 with 1 the nearer one; swapping the depths swaps the roles."""
    z1, z2 = (3.0, 2.0) if swap else (2.0, 3.0)
    c1, c2 = (0.9, 0.1, 0.3), (0.2, 0.8, 0.6)
    l1, l2 = 0.4, 1.1
    g1 = one_gaussian_kf(z1, l1, c1, z1 / 64.0)
    g2 = one_gaussian_kf(z2, l2, c2, z2 / 64.0)
    out = oracle.render(scene_of([g1, g2], [identity_view()]))[0]
    y, x = np.mgrid[0:32, 0:32]
    e = np.exp(-((x - 16.0) ** 2 + (y - 16.0) ** 2) / 2.6)
    a1 = sigmoid(l1) * e
    a2 = sigmoid(l2) * e
    a1 = np.where(a1 >= ALPHA_FLOOR, a1, 0.0)
    a2 = np.where(a2 >= ALPHA_FLOOR, a2, 0.0)
    (af, cf, zf), (ab, cb, zb) = ((a1, c1, z1), (a2, c2, z2)) if z1 < z2 else ((a2, c2, z2), (a1, c1, z1))
    for ch in range(3):
        np.testing.assert_allclose(out["rgb"][ch], af * cf[ch] + (1 - af) * ab * cb[ch], atol=1e-12)
    np.testing.assert_allclose(out["depth"], af * zf + (1 - af) * ab * zb, atol=1e-12)
    np.testing.assert_allclose(out["t_final"], (1 - af) * (1 - ab), atol=1e-12)


def test_transmittance_stop_excludes_entry():
    """Stop rule: an entry whose acceptance would take T below 1e-4 is excluded and ends
    the walk. At the centre pixel alphas are 0.99 (capped), 0.9, 0.99, 0.99 front to
    back: after two, T = 1e-3; the third would give 1e-5 < 1e-4, so exactly two
    contribute (all products well away from the threshold)."""
    l9 = math.log(0.9 / 0.1)
    kfs = [one_gaussian_kf(z, l, (1, 1, 1), z / 64.0) for z, l in ((2.0, 9.0), (2.5, l9), (3.0, 9.0), (3.5, 9.0))]
    out = oracle.render(scene_of(kfs, [identity_view()]))[0]
    assert out["n_contrib"][16, 16] == 2
    np.testing.assert_allclose(out["t_final"][16, 16], 0.01 * 0.1, rtol=1e-6)
    np.testing.assert_allclose(out["depth"][16, 16], 0.99 * 2.0 + 0.01 * 0.9 * 2.5, rtol=1e-6)


def test_invariants_and_zero_opacity(scene1):
    """A = 1 - T_final = sum of weights <= 1, T_final >= 1e-4, D' <= max z * A; with every
    opacity at zero the image is exactly the background and nothing contributes."""
    out = oracle.render(scene1)[0]
    np.testing.assert_allclose(out["alpha"], 1.0 - out["t_final"], atol=1e-12)
    assert out["t_final"].min() >= 1e-4
    assert out["alpha"].max() <= 1.0
    P = oracle.project(scene1, 0)
    assert np.all(out["depth"] <= P["t"][:, 2].max() * out["alpha"] + 1e-12)
    k = scene1.keyframes[0]
    dead = Keyframe(k.cam, k.depth, k.offset, k.rgb, np.full_like(k.logit, -60.0), k.scale)
    o = oracle.opts(bg=(0.1, 0.2, 0.3))
    out0 = oracle.render(scene_of([dead], scene1.views), o)[0]
    for ch, b in enumerate((0.1, 0.2, 0.3)):
        assert np.all(out0["rgb"][ch] == b)
    assert np.all(out0["n_contrib"] == 0) and np.all(out0["alpha"] == 0)


# ------------------------------------------------------------- brute-force pins

def _fmaf(a, b, c):
    # the float32 product is exact in float64; one float64 rounding, then one to float32
    return np.float32(float(a) * float(b) + float(c))


def _composite_python(P, order, qx, qy):
    """Per-pixel compositing written out directly: branches in float32 from the oracle's
    single-precision decision values, accumulation in float64."""
    f32 = np.float32
    T, Tf, C, D = 1.0, f32(1.0), np.zeros(3), 0.0
    last = -1
    for pos, g in enumerate(order):
        r = P[g]
        dxf, dyf = f32(r["pf"][0] - f32(qx)), f32(r["pf"][1] - f32(qy))
        a_, b_, c_ = r["conicf"]
        quad = _fmaf(a_, f32(dxf * dxf), f32(c_ * f32(dyf * dyf)))
        power = f32(f32(f32(-0.5) * quad) - f32(b_ * f32(dxf * dyf)))
        if power > 0:
            continue
        raw = f32(r["of"] * f32(math.exp(float(power))))
        alphaf = min(f32(0.99), raw)
        if alphaf < f32(1.0 / 255.0):
            continue
        test = f32(Tf * f32(f32(1.0) - alphaf))
        if test < f32(1e-4):
            break
        Tf = test
        dx, dy = r["p"][0] - qx, r["p"][1] - qy
        a64, b64, c64 = r["conic"]
        alpha = 0.99 if raw > f32(0.99) else r["o"] * math.exp(-0.5 * (a64 * dx * dx + c64 * dy * dy) - b64 * dx * dy)
        C += alpha * T * r["color"]
        D += alpha * T * r["t"][2]
        T *= 1 - alpha
        last = pos
    return C, D, T, last + 1


@pytest.mark.parametrize("seed", [11, 12])
def test_tile_lists_match_brute_force_per_pixel(seed):
    """Tiling is only a faster route to 'per pixel, every Gaussian whose tile rectangle
    contains the pixel's tile, sorted by (z rounded to f32, index)': gather that set per
    pixel from the projections, sort with Python's sort and composite pixel by pixel."""
    sc = random_scene(seed, views=((20, 18), (13, 9)))
    o = oracle.opts(tile_w=8, tile_h=8)
    outs = oracle.render(sc, o)
    for k, v in enumerate(sc.views):
        P = oracle.project(sc, k, o)
        for qy in range(v.height):
            for qx in range(v.width):
                tx, ty = qx // 8, qy // 8
                cand = [g for g in range(len(P)) if P[g]["ntiles"] > 0 and P[g]["tx0"] <= tx <= P[g]["tx1"]
                        and P[g]["ty0"] <= ty <= P[g]["ty1"]]
                cand.sort(key=lambda g: (float(np.float32(P[g]["zf"])), g))
                C, D, T, n = _composite_python(P, cand, qx, qy)
                np.testing.assert_allclose(outs[k]["rgb"][:, qy, qx], C, atol=1e-12)
                np.testing.assert_allclose(outs[k]["depth"][qy, qx], D, atol=1e-12)
                assert abs(outs[k]["t_final"][qy, qx] - T) < 1e-12
                assert outs[k]["n_contrib"][qy, qx] == n


def test_keys_match_rect_enumeration():
    """The brute-force key list (tiles x Gaussians overlap test) equals the list obtained
    by enumerating each Gaussian's tile rectangle, as a sorted multiset; its length is the
    sum of the tiles-touched counts."""
    sc = random_scene(21, views=((20, 18), (13, 9)))
    o = oracle.opts(tile_w=8, tile_h=8)
    keys, vals, _ = oracle.keys(sc, o)
    ref = []
    base = 0
    for k, v in enumerate(sc.views):
        P = oracle.project(sc, k, o)
        ntx = (v.width + 7) // 8
        for g, r in enumerate(P):
            if r["ntiles"] <= 0:
                continue
            zb = int(np.float32(r["zf"]).view(np.uint32))
            for ty in range(r["ty0"], r["ty1"] + 1):
                for tx in range(r["tx0"], r["tx1"] + 1):
                    ref.append((((base + ty * ntx + tx) << 32) | zb, g))
        base += ntx * ((v.height + 7) // 8)
    ref.sort()
    assert len(ref) == len(keys)
    assert [r[0] for r in ref] == keys.tolist()
    assert [r[1] for r in ref] == vals.tolist()


def test_square_bound_covers_every_visible_contribution_at_low_opacity():
    """With opacity <= 0.3 the alpha >= 1/255 region (radius sqrt(2 ln(255 o) lambda)) lies
    inside the 3-sigma square, so splatting over the tile lists equals splatting every
    Gaussian at every pixel with no bound at all."""
    sc = random_scene(31, views=((20, 18),), logit_mean=-2.0)
    for k in sc.keyframes:
        k.logit[:] = np.minimum(k.logit, np.float32(-0.85))     # sigmoid(-0.85) < 0.3
    o = oracle.opts(tile_w=8, tile_h=8)
    out = oracle.render(sc, o)[0]
    P = oracle.project(sc, 0, o)
    vis = [g for g in range(len(P)) if P[g]["visible"]]
    vis.sort(key=lambda g: (float(np.float32(P[g]["zf"])), g))
    for qy in range(18):
        for qx in range(20):
            C, D, T, _ = _composite_python(P, vis, qx, qy)
            np.testing.assert_allclose(out["rgb"][:, qy, qx], C, atol=1e-12)
            np.testing.assert_allclose(out["depth"][qy, qx], D, atol=1e-12)


# ------------------------------------------------------------------ adjoint pins

def _loss(scene, g):
    outs = oracle.render(scene)
    return sum(float((gi["rgb"] * o["rgb"]).sum() + (gi["depth"] * o["depth"]).sum()
                     + (gi["alpha"] * o["alpha"]).sum()) for gi, o in zip(g, outs))


def _as64(scene):
    kfs = [Keyframe(k.cam, k.depth.astype(np.float64), k.offset.astype(np.float64), k.rgb.astype(np.float64),
                    k.logit.astype(np.float64), k.scale.astype(np.float64), k.learnable) for k in scene.keyframes]
    return Scene(kfs, scene.views, scene.target_rgb, scene.target_depth, scene.depth_weight)


def test_adjoint_matches_central_differences():
    """FP64 central differences (h = 1e-6) of L = <g, render> for every scalar of the
    200-Gaussian subscene, against the oracle's hand-written adjoint: agreement to 1e-6
    relative above the FD rounding floor eps*sum|L terms|/h. A scalar whose
    perturbation changes any discrete decision (binning, accepted entries, stopping
    point) is set aside; there must be few of those."""
    from paper_2603_21055_gb300.synth import fd_subscene
    sc = _as64(fd_subscene())
    rng = np.random.default_rng(7)
    v = sc.views[0]
    g = [dict(rgb=rng.normal(size=(3, v.height, v.width)), depth=rng.normal(size=(v.height, v.width)),
              alpha=rng.normal(size=(v.height, v.width)))]
    ana = oracle.backward(sc, g)[0]
    h0 = oracle.decision_hash(sc)
    outs = oracle.render(sc)
    l_abs = sum(float(np.abs(gi[q] * o[q]).sum()) for gi, o in zip(g, outs) for q in ("rgb", "depth", "alpha"))
    kf = sc.keyframes[0]
    fields = [("offset", "d_offset", None), ("logit", "d_logit", None), ("scale", "d_scale", None),
              ("rgb", "d_rgb", 0), ("rgb", "d_rgb", 1), ("rgb", "d_rgb", 2)]
    h = 1e-6
    # rounding error of a central difference: about eps * sum|terms of L| / h
    noise = np.finfo(np.float64).eps * l_abs / h
    skipped, checked, worst = 0, 0, 0.0
    for name, gname, ch in fields:
        arr = getattr(kf, name)
        for j in range(kf.n):
            idx = (ch, j // kf.cam.width, j % kf.cam.width) if ch is not None else (j // kf.cam.width, j % kf.cam.width)
            x0 = arr[idx]
            arr[idx] = x0 + h
            lp, hp = _loss(sc, g), oracle.decision_hash(sc)
            arr[idx] = x0 - h
            lm, hm = _loss(sc, g), oracle.decision_hash(sc)
            arr[idx] = x0
            if hp != h0 or hm != h0:
                skipped += 1
                continue
            fd = (lp - lm) / (2 * h)
            an = ana[gname][idx]
            err = abs(an - fd) / (1e-6 * abs(fd) + noise)
            worst = max(worst, err)
            checked += 1
            assert err < 1.0, (name, ch, j, an, fd, noise)
    assert skipped <= 0.02 * (skipped + checked), skipped
    assert checked > 1000


def test_adjoint_sign_at_zero_and_mirror():
    """d|x|/dx = sign(x) with sign(0) = 0 (Sec. 3.2 places the Gaussian at |D + delta|):
    D + delta = -2 renders exactly like D + delta = +2, and its offset gradient has the
    opposite sign; D + delta = 0 puts the Gaussian at the keyframe centre, whose offset
    gradient is exactly zero."""
    view_c2w = np.concatenate([np.eye(3), np.array([[0.0], [0.0], [-1.0]])], 1)
    view = Camera(32, 32, 64.0, 64.0, 16.0, 16.0, pose_inverse(view_c2w).astype(np.float32))

    def sc_with(offset):
        k = one_gaussian_kf(1.0, 1.0, (0.3, 0.6, 0.9), 3.0 / 64.0)
        k.offset[:] = offset
        return scene_of([k], [view])

    rng = np.random.default_rng(5)
    g = [dict(rgb=rng.normal(size=(3, 32, 32)), depth=rng.normal(size=(32, 32)), alpha=rng.normal(size=(32, 32)))]
    a, b = sc_with(1.0), sc_with(-3.0)
    ra, rb = oracle.render(a)[0], oracle.render(b)[0]
    np.testing.assert_array_equal(ra["rgb"], rb["rgb"])
    ga, gb = oracle.backward(a, g)[0], oracle.backward(b, g)[0]
    assert ga["d_offset"][0, 0] != 0.0
    assert gb["d_offset"][0, 0] == -ga["d_offset"][0, 0]
    assert gb["d_scale"][0, 0] == ga["d_scale"][0, 0]
    z = oracle.backward(sc_with(-1.0), g)[0]
    assert z["d_offset"][0, 0] == 0.0
    assert z["d_scale"][0, 0] != 0.0


def test_contribution_magnitudes_bound_the_gradient(scene1):
    """The reported magnitude A (sum of |per-pixel contributions|) is >= |gradient| by the
    triangle inequality, and equals it when every contribution has one sign: with an
    all-positive colour gradient image, d_rgb = sum alpha T g > 0 term by term."""
    g = [dict(rgb=np.ones((3, 48, 64)), depth=np.linspace(-1, 1, 48 * 64).reshape(48, 64))]
    out = oracle.backward(scene1, g)[0]
    for q in ("d_offset", "d_rgb", "d_logit", "d_scale"):
        assert np.all(out["abs"][q] >= np.abs(out[q]) * (1 - 1e-12) - 1e-300)
    np.testing.assert_allclose(out["abs"]["d_rgb"], out["d_rgb"], rtol=1e-12)
    assert np.any(out["abs"]["d_offset"] > 1.5 * np.abs(out["d_offset"]))   # cancellation exists


def test_fixed_keyframes_get_no_gradient(scene1):
    """Eq. 1 learns only the current frame's Gaussians; neighbours are fixed (Sec. 3.2)."""
    k = scene1.keyframes[0]
    fixed = Keyframe(k.cam, k.depth, k.offset, k.rgb, k.logit, k.scale, learnable=False)
    sc = Scene([k, fixed], scene1.views, scene1.target_rgb, scene1.target_depth)
    g = [dict(rgb=np.ones((3, 48, 64)))]
    out = oracle.backward(sc, g)
    assert np.abs(out[0]["d_rgb"]).max() > 0
    assert np.all(out[1]["d_rgb"] == 0) and np.all(out[1]["d_offset"] == 0)


# --------------------------------------------------------------- loss and Adam

def test_l1_loss_closed_form():
    """Eq. 1 L1 terms as means; sign(0) = 0; invalid depth (0) is masked (U_k)."""
    v = Camera(2, 1, 1.0, 1.0, 0.0, 0.0, np.zeros((3, 4), np.float32))
    sc = Scene([], [v], [np.array([[[0.5, 0.5]], [[0.0, 1.0]], [[0.25, 0.25]]], np.float32)],
               [np.array([[2.0, 0.0]], np.float32)], depth_weight=0.1, rgb_weight=0.8)
    rend = [dict(rgb=np.array([[[0.75, 0.5]], [[0.5, 0.5]], [[0.0, 0.25]]]), depth=np.array([[1.5, 9.0]]))]
    loss, g = oracle.l1_loss(sc, rend)
    np.testing.assert_allclose(loss, 0.8 * (0.25 + 0 + 0.5 + 0.5 + 0.25 + 0) / 6 + 0.1 * 0.5 / 1, rtol=1e-15)
    np.testing.assert_allclose(g[0]["rgb"].ravel(), 0.8 / 6 * np.array([1, 0, 1, -1, -1, 0]), rtol=1e-15)
    np.testing.assert_allclose(g[0]["depth"].ravel(), [-0.1, 0.0], rtol=1e-15)


def test_adam_two_steps_closed_form():
    """Adam (bias-corrected): the first step moves by lr g/(|g| + eps); the second step
    follows from m = 0.9*0.1 g1 + 0.1 g2, v = 0.999*0.001 g1^2 + 0.001 g2^2."""
    p = np.array([1.0, -2.0, 0.5])
    g1 = np.array([0.3, -4.0, 0.0])
    g2 = np.array([-0.1, -1.0, 2.0])
    m, v = np.zeros(3), np.zeros(3)
    lr, eps = 0.01, 1e-15
    oracle.adam(p, g1.copy(), m, v, lr, eps=eps, step=1)
    np.testing.assert_allclose(p, [1.0 - 0.01, -2.0 + 0.01, 0.5], rtol=1e-14)
    oracle.adam(p, g2.copy(), m, v, lr, eps=eps, step=2)
    m2 = 0.9 * 0.1 * g1 + 0.1 * g2
    v2 = 0.999 * 0.001 * g1 ** 2 + 0.001 * g2 ** 2
    step = lr * (m2 / (1 - 0.81)) / (np.sqrt(v2 / (1 - 0.999 ** 2)) + eps)
    np.testing.assert_allclose(p, np.array([0.99, -1.99, 0.5]) - step, rtol=1e-14)


def test_pose_adjoint_matches_central_differences():
    """d L / d W for the 12 entries of the view's world->cam matrix, L = <g, render>, on
    the 200-Gaussian subscene: the oracle's adjoint against FP64 central differences of
    its own forward (h = 1e-6), above the FD rounding floor. The translation column moves
    every Gaussian, so a perturbation that changes a discrete decision is set aside; most
    entries must be checked. The reported magnitudes bound the gradient (triangle
    inequality)."""
    from paper_2603_21055_gb300.synth import fd_subscene
    sc = _as64(fd_subscene())
    v0 = sc.views[0]
    view = Camera(v0.width, v0.height, v0.fx, v0.fy, v0.cx, v0.cy, np.asarray(v0.pose, np.float64).copy())
    sc = Scene(sc.keyframes, [view], sc.target_rgb, sc.target_depth, sc.depth_weight)
    rng = np.random.default_rng(8)
    g = [dict(rgb=rng.normal(size=(3, view.height, view.width)), depth=rng.normal(size=(view.height, view.width)),
              alpha=rng.normal(size=(view.height, view.width)))]
    ana, absum = oracle.backward_pose(sc, g)
    assert np.all(absum[0] >= np.abs(ana[0]) * (1 - 1e-12))
    outs = oracle.render(sc)
    l_abs = sum(float(np.abs(gi[q] * o[q]).sum()) for gi, o in zip(g, outs) for q in ("rgb", "depth", "alpha"))
    h0 = oracle.decision_hash(sc)
    checked, worst = 0, 0.0
    for a in range(3):
        for b in range(4):
            x0 = view.pose[a, b]
            for h in (1e-6, 1e-7, 1e-8):      # a smaller step where a decision flips
                view.pose[a, b] = x0 + h
                lp, hp = _loss(sc, g), oracle.decision_hash(sc)
                view.pose[a, b] = x0 - h
                lm, hm = _loss(sc, g), oracle.decision_hash(sc)
                view.pose[a, b] = x0
                if hp == h0 and hm == h0:
                    break
            else:
                continue
            fd = (lp - lm) / (2 * h)
            noise = np.finfo(np.float64).eps * l_abs / h * 10.0
            worst = max(worst, abs(ana[0, a, b] - fd) / (1e-6 * abs(fd) + noise))
            checked += 1
    assert checked >= 10, checked
    assert worst <= 1.0, worst
