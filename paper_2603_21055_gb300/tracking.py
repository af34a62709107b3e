"""Rendering-based camera initialisation for tracking (Sec. 3.3, "Initialization").

The paper can start tracking a new frame by estimating its camera from the rendering
error of the previous frame's Gaussians against the new RGB-D frame. `PoseRefiner`
does that with the library, all on the device with no host round trip per iteration:
every iteration renders the fixed Gaussians into the view (sgad_forward), takes the
silhouette-masked L1 colour + depth loss gradient (sgad_l1_loss_grad with min_alpha),
runs the adjoint with the view-pose output (sgad_backward, d_pose = d loss / d W for the
world->cam 3x4 matrix W = [R | t]) and updates the camera (sgad_pose_adam_step): the 12
numbers are projected onto a left twist (omega, v) of the pose (W <- exp(xi) W),

    d L / d v     = sum_g d L / d t_g                   (the translation column of d L / d W)
    d L / d omega = sum_g t_g x d L / d t_g
                  = vee(R G^T - G R^T) + t x d L / d v  (G the rotation block of d L / d W)

and the twist takes an Adam step. The view itself stays at the initial pose W0; the
accumulated correction E moves the fixed Gaussians instead, by M = W0^-1 E W0 (the
keyframes' device world transform), since rendering M mu into W0 is rendering mu into
E W0. The pose estimate is E W0.

Pixels the previous frame's Gaussians do not cover render dark with no depth; left in
the loss they pull the camera towards covering more of the frame instead of towards
alignment. As in silhouette-masked tracking, the loss and its image gradients are
therefore kept only where the rendered alpha exceeds `silhouette` (0.99). The default
weights favour colour (1.0) over depth (0.1): the composited depth is not normalised by
alpha and its errors at depth discontinuities would otherwise move the minimum away from
the true pose (measured on the oracle's renders of a room).
"""
from __future__ import annotations

import math
from typing import List, Optional

import numpy as np
import torch

from . import binding as B
from . import splat


def twist_gradient(pose: np.ndarray, d_pose: np.ndarray) -> np.ndarray:
    """(d L / d omega, d L / d v) of a left perturbation exp(xi) W, from d L / d W."""
    W = np.asarray(pose, np.float64).reshape(3, 4)
    dW = np.asarray(d_pose, np.float64).reshape(3, 4)
    R, t = W[:, :3], W[:, 3]
    G, c = dW[:, :3], dW[:, 3]
    M = R @ G.T
    omega = np.array([M[1, 2] - M[2, 1], M[2, 0] - M[0, 2], M[0, 1] - M[1, 0]]) + np.cross(t, c)
    return np.concatenate([omega, c])


def exp_twist(xi: np.ndarray) -> np.ndarray:
    """4x4 rigid transform exp([omega, v]) (Rodrigues; the translation part taken as v,
    exact to first order, which is all a small step needs)."""
    w, v = np.asarray(xi[:3], np.float64), np.asarray(xi[3:], np.float64)
    th = float(np.linalg.norm(w))
    K = np.array([[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]])
    if th < 1e-12:
        R = np.eye(3) + K
    else:
        R = np.eye(3) + math.sin(th) / th * K + (1 - math.cos(th)) / th ** 2 * (K @ K)
    T = np.eye(4)
    T[:3, :3] = R
    T[:3, 3] = v
    return T


class PoseRefiner:
    """Camera of one new RGB-D frame against fixed Gaussians (typically the previous
    keyframe's). kfs: DeviceKeyframe list (their learnable flags are ignored: the
    Gaussians are not updated); camera: intrinsics and the initial world->cam pose W0;
    target_rgb (3,H,W) and target_depth (H,W): the new frame. step() only launches
    library calls on the current stream; the loss history and the pose are read back
    when asked for."""

    def __init__(self, kfs, camera, target_rgb: torch.Tensor, target_depth: torch.Tensor,
                 rgb_weight: float = 1.0, depth_weight: float = 0.1, lr_rot: float = 2e-3, lr_trans: float = 2e-3,
                 silhouette: float = 0.99):
        from .synth import Camera
        self.state = torch.zeros(B.SGAD_POSE_STATE_FLOATS, device="cuda")
        self._reset_state()
        self.kfs = [splat.DeviceKeyframe(k.cam, k.depth, k.offset, k.rgb, k.logit, k.scale, False,
                                         world_transform=self.state[12:24]) for k in kfs]
        self.cam = Camera(camera.width, camera.height, camera.fx, camera.fy, camera.cx, camera.cy,
                          np.asarray(camera.pose, np.float32).copy())
        self.W0 = np.asarray(self.cam.pose, np.float32).reshape(12).copy()
        self.trgb = [target_rgb.float().contiguous()]
        self.tdep = [target_depth.float().contiguous()]
        self.rgb_weight, self.depth_weight = rgb_weight, depth_weight
        self.silhouette = silhouette
        self.sp = splat.Splatter()
        self.images = splat.alloc_images([self.cam])
        self.d_rgb = [torch.empty_like(self.images[0]["rgb"])]
        self.d_dep = [torch.empty_like(self.images[0]["depth"])]
        self.d_pose = torch.zeros(12, device="cuda")
        self.loss = torch.zeros(1, device="cuda")
        self.valid = torch.zeros(1, dtype=torch.int32, device="cuda")
        self.lr = np.array([lr_rot, lr_trans], np.float64)
        self.sp.plan(self.kfs, [self.cam], slack=1.5)
        self._hist: List[torch.Tensor] = []

    def _reset_state(self) -> None:
        eye = torch.tensor([1.0, 0, 0, 0, 0, 1.0, 0, 0, 0, 0, 1.0, 0], device="cuda")
        self.state.zero_()
        self.state[0:12].copy_(eye)                  # E
        self.state[12:24].copy_(eye)                 # M = W0^-1 E W0

    @property
    def pose(self) -> np.ndarray:
        """Current world->cam pose estimate E W0 (3x4; reads the device state)."""
        if int(self.state[36].item()) == 0:
            return self.W0.reshape(3, 4).astype(np.float64)
        return self.state[37:49].double().cpu().numpy().reshape(3, 4)

    @property
    def history(self) -> List[float]:
        """Loss of every step's starting pose (reads the device values)."""
        return [float(x) for x in torch.cat(self._hist).cpu()] if self._hist else []

    def step(self) -> torch.Tensor:
        """One iteration; returns the (device) loss of the pose it started from."""
        views = [self.cam]
        self.sp.forward(self.kfs, views, self.images)
        self.loss.zero_()
        self.sp.l1_loss_grad(views, self.images, self.trgb, self.tdep, self.rgb_weight, self.depth_weight,
                             self.d_rgb, self.d_dep, self.loss, self.valid, min_alpha=self.silhouette)
        gin = [dict(rgb=self.d_rgb[0], depth=self.d_dep[0], pose=self.d_pose)]
        self.sp.backward(self.kfs, views, gin, [None] * len(self.kfs))
        B.sgad_pose_adam_step(self.d_pose.data_ptr(), self.W0, self.state.data_ptr(), self.lr[0], self.lr[1],
                              stream=self.sp.stream())
        loss = self.loss.clone()
        self._hist.append(loss)
        return loss[0]

    def run(self, iters: int, decay: bool = True) -> np.ndarray:
        """`iters` steps, the step size decayed by a half cosine to 5 % of its start. The
        key capacity is checked once at the end; if any forward ran out of room the
        workspace grows and the run starts again from the initial pose."""
        lr0 = self.lr.copy()
        for attempt in range(2):
            for i in range(iters):
                if decay:
                    self.lr = lr0 * (0.05 + 0.95 * 0.5 * (1.0 + math.cos(math.pi * i / max(1, iters))))
                self.step()
            self.lr = lr0
            s, _, need = self.sp.check()
            if s == 0:
                break
            self.sp.reserve(self.kfs, [self.cam], int(need * 1.5) + 4096)
            self._reset_state()
            self._hist = []
        return self.pose
