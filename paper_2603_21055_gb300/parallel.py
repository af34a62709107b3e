"""Frame-sharded mapping of an RGB-D sequence over ranks (Sec. 3.2, Eq. 1; the parallel
mapping of the runtime table and the supplementary "More Analysis").

Each frame i owns one pixel-aligned Gaussian per pixel (G_i). Mapping frame i optimises
G_i for `iters` Adam iterations of Eq. 1 against the observed colour and depth of the
views k in {i} + NN(i), NN(i) = the `nn` frames before i, rendering G_i together with the
Gaussians of those neighbours, which stay fixed (Sec. 3.2). Because a frame only needs
its own Gaussians plus already-mapped neighbours, frames can be mapped in parallel:

  * waves: frames are taken in waves of `world` consecutive frames; in wave w rank r maps
    frame w * world + r. A neighbour enters as fixed Gaussians only if it was mapped in
    an earlier wave (its parameters are then on every rank); neighbours in the same wave
    are not rendered (their views still are). After each wave one all-gather hands the
    wave's mapped parameters (offset, colour, opacity logit, scale: 6 floats per pixel)
    to every rank. With world = 1 this is the sequential mapping.
  * own_only = True: the paper's 8-GPU mode, where each frame is mapped with its own
    Gaussians alone (into the same views), so frames do not depend on one another; the
    all-gather then only assembles the mapped sequence on every rank.

Readings (the paper is silent): NN(i) = the 4 previous frames; the loss weights are the
supplementary ones (rho = 0.8, tau = 0.2, sigma = 1.0); plain initialisation offset 0,
opacity logit 0, colour = observed colour, scale = D / f. Per iteration either all views
are rendered (batched; the default) or one view, the frame's own on 40 % of the
iterations as Supp. A states and its neighbours' in turn on the others.

The data path is the library (sgad_forward, sgad_l1_loss_grad, sgad_ssim_loss_grad,
sgad_backward, sgad_adam_step_multi through `mapping.Mapper`); the exchange is
torch.distributed (NCCL between GPUs, gloo for the CPU tests of the schedule, which
replace the per-frame mapping by a stand-in function).
"""
from __future__ import annotations

import dataclasses
import time
from typing import Callable, Dict, List, Optional

import numpy as np
import torch

from . import synth

NN = 4
WEIGHTS = dict(rgb=0.8, ssim=0.2, depth=1.0)
N_PLANES = 6                       # offset, colour (3), opacity logit, scale


@dataclasses.dataclass
class Sequence:
    """An RGB-D sequence: cam -> world poses (F, 3, 4), colour (F, 3, H, W), observed
    depth (F, H, W) and the pinhole (w, h, f, cx, cy)."""
    poses: np.ndarray
    rgb: np.ndarray
    depth: np.ndarray
    size: tuple

    @property
    def n_frames(self) -> int:
        return len(self.poses)

    @property
    def hw(self) -> int:
        return int(self.size[0]) * int(self.size[1])

    def camera(self, i: int, view: bool) -> "synth.Camera":
        w, h, f, cx, cy = self.size
        p = self.poses[i]
        if view:
            p = synth._f32pose(synth.pose_inverse(np.asarray(p, np.float64)))
        return synth.Camera(int(w), int(h), float(f), float(f), float(cx), float(cy), p)


def neighbours(i: int, nn: int = NN) -> List[int]:
    return list(range(max(0, i - nn), i))


def waves(n_frames: int, world: int) -> List[List[int]]:
    return [list(range(s, min(s + world, n_frames))) for s in range(0, n_frames, world)]


def view_of_iteration(it: int, n_neighbours: int) -> int:
    """The view an iteration renders in the one-view schedule: 0 (the frame's own view)
    when it % 5 is 0 or 1, else neighbour views 1 .. n_neighbours in turn."""
    if n_neighbours == 0 or it % 5 < 2:
        return 0
    k = (it // 5) * 3 + (it % 5 - 2)
    return 1 + k % n_neighbours


def split_params(flat: torch.Tensor, h: int, w: int):
    """(offset, rgb, logit, scale) views of one frame's flat parameter vector."""
    n = h * w
    return (flat[:n].view(h, w), flat[n:4 * n].view(3, h, w), flat[4 * n:5 * n].view(h, w),
            flat[5 * n:6 * n].view(h, w))


def plain_init(seq: Sequence, i: int, device) -> torch.Tensor:
    """Flat parameters of frame i before mapping (offset 0, logit 0, observed colour,
    scale = D / f)."""
    w, h, f = int(seq.size[0]), int(seq.size[1]), np.float32(seq.size[2])
    d = np.asarray(seq.depth[i], np.float32)
    flat = np.concatenate([np.zeros(h * w, np.float32), np.asarray(seq.rgb[i], np.float32).ravel(),
                           np.zeros(h * w, np.float32), (d / f).astype(np.float32).ravel()])
    return torch.as_tensor(flat).to(device)


class FrameMapper:
    """Maps one frame of a sequence on the local GPU (library calls only)."""

    def __init__(self, seq: Sequence, nn: int = NN, iters: int = 100, weights: Optional[dict] = None,
                 tile=(16, 16), slack: float = 1.3, views_per_iter: str = "all"):
        """views_per_iter: "all" renders every view of the frame each iteration (batched);
        "one" renders one view per iteration, the frame's own view on 2 of every 5
        iterations (the 40 % of Supp. A) and its neighbours' views in turn on the rest."""
        if views_per_iter not in ("all", "one"):
            raise ValueError("views_per_iter must be 'all' or 'one'")
        self.seq, self.nn, self.iters, self.tile, self.slack = seq, nn, iters, tile, slack
        self.views_per_iter = views_per_iter
        self.weights = dict(WEIGHTS, **(weights or {}))
        self.depth = {}                                  # frame -> device depth plane
        self.losses: Dict[int, tuple] = {}               # frame -> (first, last loss with the own view)
        self.n_keyframes: Dict[int, int] = {}            # frame -> keyframes rendered (1 + fixed)
        self.psnr: Dict[int, float] = {}                 # frame -> PSNR of its own view after mapping

    def _depth(self, i: int) -> torch.Tensor:
        if i not in self.depth:
            self.depth[i] = torch.as_tensor(np.ascontiguousarray(self.seq.depth[i], np.float32)).cuda()
        return self.depth[i]

    def scene(self, i: int, fixed: Dict[int, torch.Tensor]):
        """(Scene with views {i} + NN(i), device keyframes [G_i learnable] + fixed
        neighbours present in `fixed`, flat parameters of G_i)."""
        from . import splat
        seq = self.seq
        w, h = int(seq.size[0]), int(seq.size[1])
        vids = [i] + neighbours(i, self.nn)
        views = [seq.camera(k, True) for k in vids]
        sc = synth.Scene([], views, [seq.rgb[k] for k in vids], [seq.depth[k] for k in vids],
                         depth_weight=self.weights["depth"], rgb_weight=self.weights["rgb"],
                         name="frame%d" % i, ssim_weight=self.weights["ssim"])
        flat = plain_init(seq, i, "cuda")
        off, rgb, lg, sc_ = split_params(flat, h, w)
        kfs = [splat.DeviceKeyframe(seq.camera(i, False), self._depth(i), off, rgb, lg, sc_, True)]
        for j in neighbours(i, self.nn):
            if j in fixed:
                o, r, l, s = split_params(fixed[j], h, w)
                kfs.append(splat.DeviceKeyframe(seq.camera(j, False), self._depth(j), o, r, l, s, False))
        return sc, kfs, flat

    def __call__(self, i: int, fixed: Dict[int, torch.Tensor]) -> torch.Tensor:
        from .mapping import Mapper
        for _ in range(3):
            sc, kfs, flat = self.scene(i, fixed)
            mp = Mapper(sc, tile=self.tile, slack=self.slack, kfs=kfs)
            first = last = None
            n_nb = len(sc.views) - 1
            for it in range(self.iters):
                if self.views_per_iter == "all":
                    mp.step_eager()
                    own = True
                else:
                    v = view_of_iteration(it, n_nb)
                    mp.step_views([v])
                    own = v == 0
                if own:                                  # losses of iterations that include view 0
                    last = mp.loss.clone()
                    if first is None:
                        first = last
            mp.sp.forward(mp.kfs, mp.views[:1], mp.images[:1])   # the mapped Gaussians in the own view
            if mp.ensure_capacity(self.slack):
                nan = float("nan")
                self.losses[i] = (float(first.item()) if first is not None else nan,
                                  float(last.item()) if last is not None else nan)
                self.n_keyframes[i] = len(kfs)
                mse = (mp.images[0]["rgb"].clamp(0, 1) - mp.trgb[0]).square().mean().item()
                self.psnr[i] = 10.0 * np.log10(1.0 / max(mse, 1e-12))
                return flat
            self.slack *= 1.5                           # keys outgrew the plan: redo the frame
        raise RuntimeError("frame %d: key capacity could not be met" % i)


class ShardedMapping:
    """Runs the wave schedule on this rank. `map_fn(i, fixed)` maps frame i given the
    mapped parameters of earlier frames (dict frame -> flat tensor) and returns frame i's
    flat parameters (N_PLANES * H * W floats) on `device`."""

    def __init__(self, n_frames: int, hw: int, map_fn: Callable[[int, Dict[int, torch.Tensor]], torch.Tensor],
                 own_only: bool = False, device="cuda", group=None, dtype=torch.float32):
        import torch.distributed as dist
        self.n_frames, self.hw, self.map_fn, self.own_only = n_frames, hw, map_fn, own_only
        self.dtype = dtype
        self.device = torch.device(device)
        if self.device.type == "cuda" and self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        self.group = group
        self.dist = dist.is_available() and dist.is_initialized()
        self.rank = dist.get_rank(group) if self.dist else 0
        self.world = dist.get_world_size(group) if self.dist else 1
        self.params: Dict[int, torch.Tensor] = {}
        self.wave_s: List[float] = []

    def _gather(self, mine: torch.Tensor) -> List[torch.Tensor]:
        import torch.distributed as dist
        if not self.dist:
            return [mine]
        out = [torch.empty_like(mine) for _ in range(self.world)]
        dist.all_gather(out, mine, group=self.group)
        return out

    def run(self) -> Dict[int, torch.Tensor]:
        n = N_PLANES * self.hw
        for wave in waves(self.n_frames, self.world):
            t0 = time.perf_counter()
            fixed = {} if self.own_only else self.params
            if self.rank < len(wave):
                mine = self.map_fn(wave[self.rank], fixed)
                assert mine.numel() == n and mine.device == self.device and mine.dtype == self.dtype
            else:                                        # last wave shorter than the world
                mine = torch.zeros(n, device=self.device, dtype=self.dtype)
            for j, t in zip(wave, self._gather(mine.contiguous())):
                self.params[j] = t
            if self.device.type == "cuda":
                torch.cuda.synchronize()
            self.wave_s.append(time.perf_counter() - t0)
        return self.params
