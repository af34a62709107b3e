"""Seeded synthetic RGB-D inputs for the splatting path.

This module only synthesises inputs: camera poses, ray-cast box rooms, gradient-noise
textures and the random draws of the per-Gaussian attributes. It contains none of the
splatting arithmetic (projection, binning, compositing or their adjoints); the CUDA
library and the FP64 oracle both consume the float32 arrays built here, so the two are
fed bit-identical inputs.

Conventions shared with the rest of the package:
  * pixel (u, v) has its centre at integer coordinates;
  * the ray through (u, v) is ((u - cx)/fx, (v - cy)/fy, 1) in camera space, so depth
    maps hold z-depth;
  * cameras are OpenCV-style (x right, y down, z forward);
  * keyframe poses are cam->world [R | t], view poses are world->cam [R | t], both 3x4
    row-major float32.

The workloads follow the paper's setting (Sec. 3.2: one Gaussian per keyframe pixel,
rendered into the keyframe's own view and its neighbours) with indoor depths of
0.5-6 m and TUM/Replica-like image sizes; the public datasets themselves are not used.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np

__all__ = [
    "Camera", "Keyframe", "Scene", "config1_plane", "room_scene", "config2_room",
    "config3_batching", "config4_mapping", "fd_subscene", "crop_scene", "pose_inverse",
    "rotation_about", "random_unit",
]


@dataclasses.dataclass
class Camera:
    width: int
    height: int
    fx: float
    fy: float
    cx: float
    cy: float
    pose: np.ndarray  # (3, 4) float32 (float64 allowed for finite-difference tests)

    def __post_init__(self):
        # intrinsics travel to the GPU as float32; keep exactly those values here
        self.fx, self.fy = float(np.float32(self.fx)), float(np.float32(self.fy))
        self.cx, self.cy = float(np.float32(self.cx)), float(np.float32(self.cy))

    def astuple(self):
        return (self.width, self.height, self.fx, self.fy, self.cx, self.cy,
                np.asarray(self.pose, np.float32).reshape(12))


@dataclasses.dataclass
class Keyframe:
    cam: Camera                 # pose = cam -> world
    depth: np.ndarray           # (H, W) float32, z-depth D
    offset: np.ndarray          # (H, W) float32, depth offset delta
    rgb: np.ndarray             # (3, H, W) float32
    logit: np.ndarray           # (H, W) float32, opacity logit
    scale: np.ndarray           # (H, W) float32, isotropic std-dev s in metres
    learnable: bool = True

    @property
    def n(self) -> int:
        return self.cam.width * self.cam.height


@dataclasses.dataclass
class Scene:
    keyframes: List[Keyframe]
    views: List[Camera]                     # pose = world -> cam
    target_rgb: List[np.ndarray]            # per view (3, H, W)
    target_depth: List[np.ndarray]          # per view (H, W); 0 = no valid depth
    depth_weight: float = 0.0               # weight of the L1 depth term
    rgb_weight: float = 1.0                 # weight of the L1 colour term
    name: str = ""
    ssim_weight: float = 0.0                # weight of the SSIM term (tau of Eq. 1)

    @property
    def n_gaussians(self) -> int:
        return sum(k.n for k in self.keyframes)

    @property
    def n_pixels(self) -> int:
        return sum(v.width * v.height for v in self.views)


# ----------------------------------------------------------------------------- poses

def random_unit(rng: np.random.Generator) -> np.ndarray:
    v = rng.normal(size=3)
    return v / np.linalg.norm(v)


def rotation_about(axis: np.ndarray, angle: float) -> np.ndarray:
    """Rotation matrix for `angle` radians about the unit vector `axis` (Rodrigues)."""
    a = np.asarray(axis, np.float64)
    a = a / np.linalg.norm(a)
    k = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    return np.eye(3) + math.sin(angle) * k + (1 - math.cos(angle)) * (k @ k)


def pose_inverse(pose: np.ndarray) -> np.ndarray:
    """Inverse of a rigid 3x4 transform, computed in float64."""
    p = np.asarray(pose, np.float64)
    r, t = p[:, :3], p[:, 3]
    return np.concatenate([r.T, (-r.T @ t)[:, None]], axis=1)


def _f32pose(p: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(p, np.float64).astype(np.float32))


def look_pose(position: np.ndarray, yaw: float, pitch: float) -> np.ndarray:
    """cam->world pose of a camera at `position` looking along (yaw, pitch), world z up."""
    f = np.array([math.cos(yaw) * math.cos(pitch), math.sin(yaw) * math.cos(pitch), math.sin(pitch)])
    r = np.cross(f, [0.0, 0.0, 1.0])
    r /= np.linalg.norm(r)
    d = np.cross(f, r)
    return np.concatenate([np.stack([r, d, f], axis=1), np.asarray(position, np.float64)[:, None]], axis=1)


def perturb_pose(rng, c2w: np.ndarray, max_trans: float, max_rot_deg: float,
                 exact: bool = False) -> np.ndarray:
    """Compose a cam->world pose with a random rigid perturbation.

    exact=True uses exactly `max_trans` / `max_rot_deg`; otherwise both are drawn
    uniformly in [0, max]."""
    t_mag = max_trans if exact else rng.uniform(0.0, max_trans)
    a_mag = math.radians(max_rot_deg if exact else rng.uniform(0.0, max_rot_deg))
    dt = random_unit(rng) * t_mag
    dr = rotation_about(random_unit(rng), a_mag)
    r = c2w[:, :3] @ dr
    return np.concatenate([r, (c2w[:, 3] + dt)[:, None]], axis=1)


# ------------------------------------------------------------------ config 1: plane

def config1_plane(seed: int = 1, width: int = 64, height: int = 48, f: float = 60.0) -> Scene:
    """Tiny plain-method case: one keyframe on a tilted plane, one nearby view.

    Inverse depth is affine in (u, v) with z = 0.5 m at (0, 0) and 3.0 m at the far
    corner, plus N(0, 1 cm) noise; delta ~ N(0, 2 cm), RGB ~ U[0, 1], opacity logits
    ~ N(1, 0.5) and scale = D/fx * U[0.8, 1.2] (the r = D/F initialisation of the paper's
    implementation details). The view is the keyframe pose moved by 3 cm along a seeded
    direction and turned by 1 degree about a seeded axis; the target is a seeded U[0, 1]
    image (colour L1 only)."""
    rng = np.random.default_rng(seed)
    u = np.arange(width, dtype=np.float64)[None, :]
    v = np.arange(height, dtype=np.float64)[:, None]
    inv = 2.0 + (1.0 / 3.0 - 2.0) * (u / (width - 1) + v / (height - 1)) / 2.0
    depth = (1.0 / inv + rng.normal(0.0, 0.01, size=(height, width))).astype(np.float32)
    offset = rng.normal(0.0, 0.02, size=(height, width)).astype(np.float32)
    rgb = rng.uniform(0.0, 1.0, size=(3, height, width)).astype(np.float32)
    logit = rng.normal(1.0, 0.5, size=(height, width)).astype(np.float32)
    scale = (depth / np.float32(f) * rng.uniform(0.8, 1.2, size=(height, width))).astype(np.float32)
    kf_pose = np.concatenate([np.eye(3), np.zeros((3, 1))], axis=1)
    cam = Camera(width, height, f, f, width / 2.0, height / 2.0, _f32pose(kf_pose))
    view_c2w = perturb_pose(rng, kf_pose, 0.03, 1.0, exact=True)
    view = Camera(width, height, f, f, width / 2.0, height / 2.0, _f32pose(pose_inverse(view_c2w)))
    target = rng.uniform(0.0, 1.0, size=(3, height, width)).astype(np.float32)
    return Scene([Keyframe(cam, depth, offset, rgb, logit, scale)], [view], [target],
                 [np.zeros((height, width), np.float32)], depth_weight=0.0, name="plane64x48")


# --------------------------------------------------------------- box room ray caster

@dataclasses.dataclass
class Room:
    shell_hi: np.ndarray
    boxes_lo: np.ndarray          # (B, 3)
    boxes_hi: np.ndarray          # (B, 3)
    face_color: np.ndarray        # (6 * (B + 1), 3): shell faces first, then 6 per box
    grads: np.ndarray             # (P, P, P, 3, 3) unit gradients, one per RGB channel
    noise_freq: float


def make_room(rng: np.random.Generator, n_boxes: int = 20, shell=(6.0, 5.0, 3.0),
              keep_free: Optional[Tuple[np.ndarray, float]] = None) -> Room:
    """A 6x5x3 m shell with `n_boxes` axis-aligned boxes (edges U[0.2, 1.5] m), half of
    them standing on the floor. Boxes intersecting the sphere `keep_free` (centre,
    radius) are redrawn, so cameras inside it see every surface at >= 0.5 m."""
    hi = np.asarray(shell, np.float64)
    lo_l, hi_l = [], []
    while len(lo_l) < n_boxes:
        size = rng.uniform(0.2, 1.5, size=3)
        size = np.minimum(size, hi - 0.05)
        x = rng.uniform(0.0, hi[0] - size[0])
        y = rng.uniform(0.0, hi[1] - size[1])
        z = 0.0 if rng.uniform() < 0.5 else rng.uniform(0.0, hi[2] - size[2])
        blo = np.array([x, y, z])
        bhi = blo + size
        if keep_free is not None:
            c, rad = keep_free
            nearest = np.clip(c, blo, bhi)
            if np.linalg.norm(nearest - c) < rad:
                continue
        lo_l.append(blo)
        hi_l.append(bhi)
    face_color = rng.uniform(0.15, 0.85, size=(6 * (n_boxes + 1), 3))
    p = 32
    g = rng.normal(size=(p, p, p, 3, 3))
    g = (g / np.linalg.norm(g, axis=-1, keepdims=True)).astype(np.float32)
    return Room(hi, np.array(lo_l), np.array(hi_l), face_color, g, 1.0)


def _fade(t):
    return t * t * t * (t * (t * 6.0 - 15.0) + 10.0)


def gradient_noise(room: Room, pts: np.ndarray) -> np.ndarray:
    """Smooth lattice gradient noise, three independent channels, roughly in [-1, 1], at
    points (N, 3): quintic interpolation of dot products with seeded unit gradients at
    the 8 cell corners. Returns (N, 3)."""
    p = room.grads.shape[0]
    table = room.grads.reshape(p * p * p, 3, 3)
    i0 = np.floor(pts).astype(np.int64)
    f = (pts - i0).astype(np.float32)
    w = _fade(f)
    out = np.zeros((pts.shape[0], 3), np.float32)
    for cx in (0, 1):
        ix = ((i0[:, 0] + cx) % p) * (p * p)
        wx = w[:, 0] if cx else 1.0 - w[:, 0]
        dx = f[:, 0] - cx
        for cy in (0, 1):
            ixy = ix + ((i0[:, 1] + cy) % p) * p
            wxy = wx * (w[:, 1] if cy else 1.0 - w[:, 1])
            dy = f[:, 1] - cy
            for cz in (0, 1):
                g = table[ixy + (i0[:, 2] + cz) % p]           # (N, 3 channels, 3)
                wxyz = wxy * (w[:, 2] if cz else 1.0 - w[:, 2])
                dz = f[:, 2] - cz
                dot = g[:, :, 0] * dx[:, None] + g[:, :, 1] * dy[:, None] + g[:, :, 2] * dz[:, None]
                out += wxyz[:, None] * dot
    return out * 1.5


def shade(room: Room, pts: np.ndarray, face: np.ndarray) -> np.ndarray:
    """RGB in [0, 1] of surface points: per-face base colour plus three octaves of
    gradient noise (base frequency ~1 per metre), one independent field per channel."""
    q = pts * room.noise_freq
    n = gradient_noise(room, q) + 0.5 * gradient_noise(room, 2.0 * q) + 0.25 * gradient_noise(room, 4.0 * q)
    out = room.face_color[face].T + 0.3 * n.T
    return np.clip(out, 0.0, 1.0)


def raycast(room: Room, c2w: np.ndarray, width: int, height: int, fx: float, fy: float,
            cx: float, cy: float) -> Tuple[np.ndarray, np.ndarray]:
    """Ray-cast a pinhole camera into the room; returns z-depth (H, W) and RGB (3, H, W)."""
    c2w = np.asarray(c2w, np.float64)
    u, v = np.meshgrid(np.arange(width, dtype=np.float64), np.arange(height, dtype=np.float64))
    rc = np.stack([(u - cx) / fx, (v - cy) / fy, np.ones_like(u)], axis=-1).reshape(-1, 3)
    d = rc @ c2w[:, :3].T
    o = c2w[:, 3]
    dx, dy, dz = d[:, 0], d[:, 1], d[:, 2]
    with np.errstate(divide="ignore", invalid="ignore"):
        ix, iy, iz = 1.0 / dx, 1.0 / dy, 1.0 / dz
        # inside of the shell: leave through the nearest wall (face = 2 * axis + side)
        best_t = np.full(d.shape[0], np.inf)
        best_face = np.zeros(d.shape[0], np.int64)
        for a, (da, ia) in enumerate(((dx, ix), (dy, iy), (dz, iz))):
            t = np.where(da > 0, (room.shell_hi[a] - o[a]) * ia, np.where(da < 0, -o[a] * ia, np.inf))
            better = t < best_t
            best_t = np.where(better, t, best_t)
            best_face = np.where(better, 2 * a + (da > 0), best_face)
        for b in range(room.boxes_lo.shape[0]):
            lo, hi = room.boxes_lo[b], room.boxes_hi[b]
            tmins, tmaxs = [], []
            for a, ia in enumerate((ix, iy, iz)):
                t1 = (lo[a] - o[a]) * ia
                t2 = (hi[a] - o[a]) * ia
                tmins.append(np.minimum(t1, t2))
                tmaxs.append(np.maximum(t1, t2))
            tnear = np.maximum(np.maximum(tmins[0], tmins[1]), tmins[2])
            tfar = np.minimum(np.minimum(tmaxs[0], tmaxs[1]), tmaxs[2])
            hit = (tnear <= tfar) & (tnear > 1e-6) & (tnear < best_t)
            if np.any(hit):
                ax = np.where(tmins[0] >= tmins[1], np.where(tmins[0] >= tmins[2], 0, 2),
                              np.where(tmins[1] >= tmins[2], 1, 2))
                da = np.choose(ax, (dx, dy, dz))
                best_t = np.where(hit, tnear, best_t)
                best_face = np.where(hit, 6 * (b + 1) + ax * 2 + (da < 0), best_face)
    pts = o + d * best_t[:, None]
    rgb = shade(room, pts, best_face)
    depth = best_t.reshape(height, width)          # r_cam has z = 1, so t is z-depth
    return depth.astype(np.float32), rgb.reshape(3, height, width).astype(np.float32)


def keyframe_path(rng: np.random.Generator, n: int, centre: np.ndarray, step: float = 0.10,
                  turn_deg: float = 5.0) -> List[np.ndarray]:
    """cam->world poses on a smooth seeded path: ~`step` m and ~`turn_deg` apart, at
    1.2-1.8 m height, looking roughly horizontally at the walls."""
    pos = centre + np.array([rng.uniform(-0.2, 0.2), rng.uniform(-0.2, 0.2), 0.0])
    pos[2] = rng.uniform(1.3, 1.7)
    yaw = rng.uniform(0.0, 2.0 * math.pi)
    pitch = math.radians(rng.uniform(-8.0, 8.0))
    heading = rng.uniform(0.0, 2.0 * math.pi)
    poses = []
    for _ in range(n):
        poses.append(look_pose(pos, yaw, pitch))
        heading += rng.normal(0.0, 0.3)
        pos = pos + step * np.array([math.cos(heading), math.sin(heading), rng.normal(0.0, 0.2)])
        pos[2] = float(np.clip(pos[2], 1.2, 1.8))
        if np.linalg.norm(pos[:2] - centre[:2]) > 0.35:     # stay in the free region
            heading += math.pi
            pos[:2] = centre[:2] + 0.35 * (pos[:2] - centre[:2]) / np.linalg.norm(pos[:2] - centre[:2])
        yaw += math.radians(turn_deg) * (1.0 if rng.uniform() < 0.8 else -1.0)
        pitch = float(np.clip(pitch + math.radians(rng.normal(0.0, 1.0)), -0.2, 0.2))
    return poses


def room_scene(seed: int, n_keyframes: int, keyframe_size: Tuple[int, int, float, float, float],
               view_sizes: Sequence[Tuple[int, int, float, float, float]],
               view_of_keyframe: Optional[Sequence[int]] = None,
               max_trans: float = 0.05, max_rot_deg: float = 2.0, offset_std: float = 0.03,
               depth_weight: float = 0.1, name: str = "") -> Scene:
    """Keyframes and views in a seeded box room.

    keyframe_size and each entry of view_sizes are (W, H, f, cx, cy). View j is keyframe
    `view_of_keyframe[j]`'s pose perturbed by <= max_trans m and <= max_rot_deg degrees
    (default: j mod n_keyframes). Keyframe depth and RGB are ray-cast; delta ~ N(0,
    offset_std), logit ~ N(1, 0.5), scale = D/fx * U[0.8, 1.2]. View targets are the
    ray-cast RGB-D at the view pose."""
    rng = np.random.default_rng(seed)
    centre = np.array([3.0, 2.5, 1.5])
    room = make_room(rng, keep_free=(centre, 1.1))
    poses = keyframe_path(rng, n_keyframes, centre)
    kw, kh, kf_f, kcx, kcy = keyframe_size
    kfs = []
    for p in poses:
        depth, rgb = raycast(room, p, kw, kh, kf_f, kf_f, kcx, kcy)
        offset = rng.normal(0.0, offset_std, size=(kh, kw)).astype(np.float32)
        logit = rng.normal(1.0, 0.5, size=(kh, kw)).astype(np.float32)
        scale = (depth / np.float32(kf_f) * rng.uniform(0.8, 1.2, size=(kh, kw))).astype(np.float32)
        kfs.append(Keyframe(Camera(kw, kh, kf_f, kf_f, kcx, kcy, _f32pose(p)), depth, offset, rgb, logit, scale))
    views, trgb, tdep = [], [], []
    for j, (vw, vh, vf, vcx, vcy) in enumerate(view_sizes):
        k = view_of_keyframe[j] if view_of_keyframe is not None else j % n_keyframes
        c2w = perturb_pose(rng, poses[k], max_trans, max_rot_deg)
        depth, rgb = raycast(room, c2w, vw, vh, vf, vf, vcx, vcy)
        views.append(Camera(vw, vh, vf, vf, vcx, vcy, _f32pose(pose_inverse(c2w))))
        trgb.append(rgb)
        tdep.append(depth)
    return Scene(kfs, views, trgb, tdep, depth_weight=depth_weight, name=name)


VGA = (640, 480, 600.0, 320.0, 240.0)
QVGA = (320, 240, 300.0, 160.0, 120.0)
REPLICA = (1200, 680, 600.0, 600.0, 340.0)


def config2_room(seed: int = 2) -> Scene:
    """Paper-shaped plain-method workload: 8 keyframes at 640x480 (2,457,600 Gaussians)
    rendered into 8 neighbouring views (<= 5 cm / <= 2 degrees from the keyframes),
    fx = fy = 600, L1 colour + 0.1 L1 depth."""
    return room_scene(seed, 8, VGA, [VGA] * 8, name="room8x640x480")


def config3_batching(seed: int = 3) -> Scene:
    """Batching workload: 16 keyframes at 640x480 (4,915,200 Gaussians) into 32 views of
    uneven size: 8 at 320x240 (fx 300), 16 at 640x480 (fx 600), 8 at 1200x680 (fx 600)."""
    sizes = [QVGA] * 8 + [VGA] * 16 + [REPLICA] * 8
    return room_scene(seed, 16, VGA, sizes, view_of_keyframe=[j % 16 for j in range(32)],
                      name="room16kf_32views_uneven")


def batching_small(seed: int = 6) -> Scene:
    """A small version of the batching workload for parity tests: 2 keyframes of 160x120
    (fx 150) into 5 views of uneven size and ragged tile edges: 2 at 72x54 (fx 67.5),
    2 at 160x120 (fx 150) and 1 at 300x170 (fx 150, cx 150, cy 85)."""
    small = (72, 54, 67.5, 36.0, 27.0)
    mid = (160, 120, 150.0, 80.0, 60.0)
    wide = (300, 170, 150.0, 150.0, 85.0)
    return room_scene(seed, 2, mid, [small, small, mid, mid, wide], view_of_keyframe=[0, 1, 0, 1, 0],
                      name="room2kf_5views_uneven")


def config4_mapping(seed: int = 4) -> Scene:
    """Mapping workload: 10 keyframes at 1200x680 (8,160,000 Gaussians) and 10 views at
    the keyframe poses themselves (no perturbation)."""
    return room_scene(seed, 10, REPLICA, [REPLICA] * 10, max_trans=0.0, max_rot_deg=0.0,
                      name="room10x1200x680")


def crop_scene(scene: Scene, kf_box: Tuple[int, int, int, int], view_box: Tuple[int, int, int, int],
               n_keyframes: Optional[int] = None, n_views: Optional[int] = None) -> Scene:
    """A smaller case cut out of a room scene: every keyframe is cropped to the pixel box
    (x0, y0, w, h) (principal point shifted accordingly) and every view to view_box."""
    kx, ky, kw, kh = kf_box
    vx, vy, vw, vh = view_box
    kfs = []
    for k in scene.keyframes[: n_keyframes or len(scene.keyframes)]:
        c = k.cam
        cam = Camera(kw, kh, c.fx, c.fy, c.cx - kx, c.cy - ky, c.pose.copy())
        sl = (slice(ky, ky + kh), slice(kx, kx + kw))
        kfs.append(Keyframe(cam, np.ascontiguousarray(k.depth[sl]), np.ascontiguousarray(k.offset[sl]),
                            np.ascontiguousarray(k.rgb[(slice(None),) + sl]),
                            np.ascontiguousarray(k.logit[sl]), np.ascontiguousarray(k.scale[sl]), k.learnable))
    views, tr, td = [], [], []
    nv = n_views or len(scene.views)
    for c, r, d in zip(scene.views[:nv], scene.target_rgb[:nv], scene.target_depth[:nv]):
        views.append(Camera(vw, vh, c.fx, c.fy, c.cx - vx, c.cy - vy, c.pose.copy()))
        sl = (slice(vy, vy + vh), slice(vx, vx + vw))
        tr.append(np.ascontiguousarray(r[(slice(None),) + sl]))
        td.append(np.ascontiguousarray(d[sl]))
    return Scene(kfs, views, tr, td, scene.depth_weight, scene.rgb_weight, scene.name + "_crop",
                 scene.ssim_weight)


def fd_subscene(seed: int = 5, kw: int = 20, kh: int = 10, vw: int = 32, vh: int = 32) -> Scene:
    """200 Gaussians (a 20x10 keyframe) rendered into a 32x32 view, focal length scaled
    so the keyframe's content fills the view; used for finite-difference checks."""
    rng = np.random.default_rng(seed)
    f = 40.0
    u = np.arange(kw, dtype=np.float64)[None, :]
    v = np.arange(kh, dtype=np.float64)[:, None]
    depth = (1.5 + 0.02 * u + 0.03 * v + rng.normal(0.0, 0.01, size=(kh, kw))).astype(np.float32)
    offset = rng.normal(0.0, 0.02, size=(kh, kw)).astype(np.float32)
    rgb = rng.uniform(0.0, 1.0, size=(3, kh, kw)).astype(np.float32)
    logit = rng.normal(0.0, 0.5, size=(kh, kw)).astype(np.float32)
    scale = (depth / np.float32(f) * rng.uniform(1.5, 2.5, size=(kh, kw))).astype(np.float32)
    kf_pose = np.concatenate([np.eye(3), np.zeros((3, 1))], axis=1)
    cam = Camera(kw, kh, f, f, (kw - 1) / 2.0, (kh - 1) / 2.0, _f32pose(kf_pose))
    view_c2w = perturb_pose(rng, kf_pose, 0.02, 1.0, exact=True)
    vf = f * 1.4
    view = Camera(vw, vh, vf, vf, (vw - 1) / 2.0, (vh - 1) / 2.0, _f32pose(pose_inverse(view_c2w)))
    target = rng.uniform(0.0, 1.0, size=(3, vh, vw)).astype(np.float32)
    tdepth = (1.5 + rng.normal(0.0, 0.05, size=(vh, vw))).astype(np.float32)
    return Scene([Keyframe(cam, depth, offset, rgb, logit, scale)], [view], [target], [tdepth],
                 depth_weight=0.1, name="fd20x10_to32x32")
