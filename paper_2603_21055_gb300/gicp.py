"""Geometric tracking on the GPU (Sec. 3.3, Eq. 2) over the library's C ABI
(include/sgad_gicp.h): geometry Gaussians of each depth frame, GICP of the frame against
the global set T, and T's update with the frame's non-overlapping Gaussians.

`GaussianSet` holds one set in device memory (torch tensors; the library writes them);
`GicpTracker` owns the workspace and runs frame -> track -> insert. With the constant
speed initialisation of Sec. 3.3, the first guess of frame i is
W_{i-1} W_{i-2}^-1 W_{i-1} (cam -> world); `track_sequence` does that for a list of
depth frames.
"""
from __future__ import annotations

from typing import List, Optional

import numpy as np
import torch

from . import binding as B


class GaussianSet:
    def __init__(self, capacity: int, device="cuda"):
        self.capacity = int(capacity)
        self.pos = torch.zeros(self.capacity, 4, device=device)
        self.cov = torch.zeros(self.capacity, 8, device=device)
        self.normal = torch.zeros(self.capacity, 4, device=device)
        self.count = torch.zeros(1, dtype=torch.int32, device=device)
        self.c = B.sgad_gaussian_set(self.pos.data_ptr(), self.cov.data_ptr(), self.normal.data_ptr(),
                                     self.count.data_ptr(), self.capacity)

    def n(self) -> int:
        return int(self.count.item())

    def load(self, pos: np.ndarray, cov: np.ndarray, normal: np.ndarray) -> None:
        """Fill from host arrays: pos (n, 3), cov (n, 3, 3) symmetric, normal (n, 3)."""
        n = len(pos)
        assert n <= self.capacity
        p = np.zeros((n, 4), np.float32)
        p[:, :3] = pos
        c = np.zeros((n, 8), np.float32)
        cv = np.asarray(cov, np.float64)
        c[:, 0], c[:, 1], c[:, 2], c[:, 3], c[:, 4], c[:, 5] = (cv[:, 0, 0], cv[:, 0, 1], cv[:, 0, 2], cv[:, 1, 1],
                                                                cv[:, 1, 2], cv[:, 2, 2])
        nr = np.zeros((n, 4), np.float32)
        nr[:, :3] = normal
        self.pos[:n] = torch.as_tensor(p)
        self.cov[:n] = torch.as_tensor(c)
        self.normal[:n] = torch.as_tensor(nr)
        self.count.fill_(n)

    def host(self):
        """(pos (n,3), cov (n,3,3), normal (n,3)) as numpy."""
        n = self.n()
        p = self.pos[:n, :3].cpu().numpy()
        c = self.cov[:n].cpu().numpy().astype(np.float64)
        C = np.empty((n, 3, 3))
        C[:, 0, 0], C[:, 0, 1], C[:, 0, 2] = c[:, 0], c[:, 1], c[:, 2]
        C[:, 1, 0], C[:, 1, 1], C[:, 1, 2] = c[:, 1], c[:, 3], c[:, 4]
        C[:, 2, 0], C[:, 2, 1], C[:, 2, 2] = c[:, 2], c[:, 4], c[:, 5]
        return p, C, self.normal[:n, :3].cpu().numpy()


def pose44(P) -> np.ndarray:
    T = np.eye(4)
    T[:3] = np.asarray(P, np.float64).reshape(3, 4)
    return T


class GicpTracker:
    def __init__(self, params: Optional[B.sgad_gicp_params] = None, src_capacity: int = 1 << 16,
                 map_capacity: int = 1 << 20, **overrides):
        self.p = params or B.sgad_gicp_default_params()
        for k, v in overrides.items():
            setattr(self.p, k, v)
        self.p.src_capacity, self.p.map_capacity = int(src_capacity), int(map_capacity)
        self.src = GaussianSet(src_capacity)
        self.map = GaussianSet(map_capacity)
        self.ws_bytes = B.sgad_gicp_workspace_size(self.p)
        self.ws = torch.zeros(self.ws_bytes, dtype=torch.uint8, device="cuda")
        self.pix = torch.empty(src_capacity, dtype=torch.int32, device="cuda")

    def stream(self) -> int:
        return torch.cuda.current_stream().cuda_stream

    def frame(self, cam, depth: torch.Tensor, knn_out: Optional[torch.Tensor] = None) -> None:
        """T_i of a depth frame (device (H, W) FP32) into self.src."""
        assert depth.is_cuda and depth.dtype == torch.float32 and depth.is_contiguous()
        c = B.sgad_camera(cam.width, cam.height, cam.fx, cam.fy, cam.cx, cam.cy)
        B.sgad_gicp_frame(self.p, c, depth.data_ptr(), self.src.c, self.pix.data_ptr(),
                          knn_out.data_ptr() if knn_out is not None else 0, self.ws.data_ptr(), self.ws_bytes,
                          self.stream())

    def index(self) -> None:
        B.sgad_gicp_index(self.p, self.map.c, self.ws.data_ptr(), self.ws_bytes, self.stream())

    def correspond(self, pose, idx_out: torch.Tensor) -> None:
        B.sgad_gicp_correspond(self.p, self.src.c, self.map.c, np.asarray(pose, np.float32).ravel(),
                               idx_out.data_ptr(), self.ws.data_ptr(), self.ws_bytes, self.stream())

    def linearize(self, pose) -> np.ndarray:
        out = torch.zeros(29, dtype=torch.float64, device="cuda")
        B.sgad_gicp_linearize(self.p, self.src.c, self.map.c, np.asarray(pose, np.float32).ravel(), out.data_ptr(),
                              self.ws.data_ptr(), self.ws_bytes, self.stream())
        return out.cpu().numpy()

    def set_pose(self, pose) -> None:
        B.sgad_gicp_set_pose(np.asarray(pose, np.float64).ravel(), self.ws.data_ptr(), self.ws_bytes, self.stream())

    def track(self, pose0=None) -> None:
        """GICP from pose0 (cam -> world 3x4), or from the workspace's pose when None."""
        p0 = np.asarray(pose0, np.float64).ravel() if pose0 is not None else None
        B.sgad_gicp_track(self.p, self.src.c, self.map.c, p0, self.ws.data_ptr(), self.ws_bytes, self.stream())

    def capture(self, cam, height: int, width: int) -> None:
        """Records one frame's library calls (geometry Gaussians of self.depth_in, GICP from
        the workspace's pose, map update) as a CUDA graph; `step` replays it."""
        self.cam = cam
        self.depth_in = torch.zeros(height, width, device="cuda")
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):                 # warm-up outside the capture
            self.frame(cam, self.depth_in)
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self.frame(cam, self.depth_in)
            self.track(None)
            self.insert()

    def step(self, depth: torch.Tensor, guess) -> None:
        """One frame through the captured graph: copy the depth in, set the starting pose,
        replay (frame -> GICP -> map update)."""
        self.depth_in.copy_(depth)
        self.set_pose(guess)
        self.graph.replay()

    def insert(self) -> None:
        B.sgad_gicp_insert(self.p, self.src.c, self.map.c, self.ws.data_ptr(), self.ws_bytes, self.stream())

    def result(self):
        pose, st = B.sgad_gicp_result(self.ws.data_ptr(), self.ws_bytes, self.stream())
        return np.asarray(pose).reshape(3, 4), st

    def track_sequence(self, cam, depths: List[torch.Tensor], first_pose) -> List[np.ndarray]:
        """Cam -> world poses of a depth sequence: frame 0 at `first_pose` seeds the map;
        every later frame starts from the constant-speed guess, is tracked by GICP and
        then adds its non-overlapping Gaussians to the map."""
        poses = [np.asarray(first_pose, np.float64).reshape(3, 4)]
        self.frame(cam, depths[0])
        self.set_pose(poses[0])
        self.insert()
        for i in range(1, len(depths)):
            if i >= 2:
                T1, T0 = pose44(poses[-1]), pose44(poses[-2])
                guess = (T1 @ np.linalg.inv(T0) @ T1)[:3]
            else:
                guess = poses[-1]
            self.frame(cam, depths[i])
            self.track(guess)
            self.insert()
            pose, _ = self.result()
            poses.append(pose)
        return poses
