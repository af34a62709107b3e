"""Torch-facing wrappers of the splatting library.

`Splatter` owns a library context and a workspace tensor and calls the C ABI with
device pointers of torch tensors on the current CUDA stream. `SplatFn` exposes the
hand-written adjoint as a torch.autograd.Function: its forward is sgad_forward, its
backward sgad_backward (transmittance recomputed by division, nothing but the final
transmittance and contributor count stored per pixel).
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass
from typing import List, Optional, Sequence

import numpy as np
import torch

from . import binding as B


def _cam(c) -> B.sgad_camera:
    pose = np.asarray(c.pose, np.float32).reshape(12)
    return B.sgad_camera(int(c.width), int(c.height), float(c.fx), float(c.fy), float(c.cx), float(c.cy),
                         (C.c_float * 12)(*pose.tolist()))


def _ptr(t: Optional[torch.Tensor]) -> int:
    if t is None:
        return 0
    assert t.is_cuda and t.is_contiguous() and t.dtype == torch.float32, "FP32 contiguous CUDA tensor expected"
    return t.data_ptr()


@dataclass
class DeviceKeyframe:
    cam: object                      # synth.Camera-like (cam -> world)
    depth: torch.Tensor              # (H, W)
    offset: torch.Tensor             # (H, W)
    rgb: torch.Tensor                # (3, H, W)
    logit: torch.Tensor              # (H, W)
    scale: torch.Tensor              # (H, W)
    learnable: bool = True
    world_transform: Optional[torch.Tensor] = None   # (12,) device 3x4 applied to the centres (fixed keyframes)

    @property
    def n(self) -> int:
        return self.cam.width * self.cam.height


def upload_keyframes(scene, device="cuda") -> List[DeviceKeyframe]:
    out = []
    for k in scene.keyframes:
        f = lambda a: torch.as_tensor(np.ascontiguousarray(a, np.float32)).to(device)
        out.append(DeviceKeyframe(k.cam, f(k.depth), f(k.offset), f(k.rgb), f(k.logit), f(k.scale),
                                  bool(k.learnable)))
    return out


def upload_targets(scene, device="cuda"):
    f = lambda a: torch.as_tensor(np.ascontiguousarray(a, np.float32)).to(device)
    return [f(r) for r in scene.target_rgb], [f(d) for d in scene.target_depth]


def upload_window(scene, device="cuda"):
    """The keyframes, the targets and a loss slot of one mapping window as views of one
    flat FP32 device buffer, each array starting on a 256-byte boundary, laid out as
    [per keyframe: offset, rgb, logit, scale] [loss] [per keyframe: depth] [per view:
    target rgb, target depth]. What a mapping step updates is the prefix of `n_state`
    floats, so moving a window between host and device takes one copy each way.
    Returns (buffer, n_state, keyframes, target_rgb, target_depth, loss)."""
    state = [(k, n) for k in scene.keyframes for n in ("offset", "rgb", "logit", "scale")]
    rest = [(k, "depth") for k in scene.keyframes]
    arrays = [np.ascontiguousarray(getattr(k, n), np.float32) for k, n in state]
    arrays.append(np.zeros(1, np.float32))                               # loss
    arrays += [np.ascontiguousarray(k.depth, np.float32) for k, _ in rest]
    arrays += [np.ascontiguousarray(a, np.float32) for a in scene.target_rgb]
    arrays += [np.ascontiguousarray(a, np.float32) for a in scene.target_depth]
    offs, n = [], 0
    for a in arrays:
        offs.append(n)
        n += (a.size + 63) // 64 * 64
    host = np.zeros(n, np.float32)
    for a, o in zip(arrays, offs):
        host[o:o + a.size] = a.ravel()
    buf = torch.as_tensor(host).to(device)
    views = [buf[o:o + a.size].view(a.shape) for a, o in zip(arrays, offs)]
    n_state = offs[len(state)] + 64
    ns = len(state)
    kfs = []
    for i, k in enumerate(scene.keyframes):
        off, rgb, logit, scale = views[4 * i:4 * i + 4]
        kfs.append(DeviceKeyframe(k.cam, views[ns + 1 + i], off, rgb, logit, scale, bool(k.learnable)))
    nk, nv = len(scene.keyframes), len(scene.views)
    trgb = views[ns + 1 + nk:ns + 1 + nk + nv]
    tdep = views[ns + 1 + nk + nv:ns + 1 + nk + 2 * nv]
    return buf, n_state, kfs, trgb, tdep, views[ns]


def _schedule(x) -> int:
    if isinstance(x, str):
        names = {v: k for k, v in B.SCHEDULE_NAMES.items()}
        if x not in names:
            raise ValueError("schedule must be one of %s" % sorted(names))
        return names[x]
    return int(x)


def alloc_images(views, device="cuda"):
    return [dict(rgb=torch.empty(3, v.height, v.width, device=device),
                 depth=torch.empty(v.height, v.width, device=device),
                 alpha=torch.empty(v.height, v.width, device=device)) for v in views]


class Splatter:
    """A library context plus a workspace sized for one problem shape."""

    def __init__(self, tile=(16, 16), bg=(0.0, 0.0, 0.0), sort_smem_cap: int = 0, freeze_offset: bool = False,
                 fwd_batch: int = 0, bwd_batch: int = 0, fwd_schedule="tiles", bwd_schedule="tiles",
                 bwd_algorithm: str = "warp_local", max_blocks: int = 0, options=None):
        """options: a complete sgad_options (e.g. another Splatter's tuned options), used
        instead of the other arguments. max_blocks caps the persistent grid (0: as many
        blocks as are resident)."""
        if options is not None:
            o = B.sgad_options.from_buffer_copy(options)
        else:
            o = B.sgad_default_options()
            o.tile_w, o.tile_h = int(tile[0]), int(tile[1])
            for i in range(3):
                o.bg[i] = float(bg[i])
            o.sort_smem_cap = int(sort_smem_cap)
            o.freeze_offset = int(bool(freeze_offset))
            if fwd_batch:
                o.fwd_batch = int(fwd_batch)
            if bwd_batch:
                o.bwd_batch = int(bwd_batch)
            o.fwd_schedule = _schedule(fwd_schedule)
            o.bwd_schedule = _schedule(bwd_schedule)
            o.bwd_algorithm = {"pairs": B.SGAD_BWD_PAIRS, "warp_reduce": B.SGAD_BWD_WARP_REDUCE,
                               "warp_local": B.SGAD_BWD_WARP_LOCAL}[bwd_algorithm]
            o.max_blocks = int(max_blocks)
        self.options = o
        self.ctx = B.sgad_create(o)
        self.workspace: Optional[torch.Tensor] = None
        self.key_capacity = 0
        self._cache = {}
        self._ssim_ws: Optional[torch.Tensor] = None

    def __del__(self):
        try:
            if getattr(self, "ctx", None):
                B.sgad_destroy(self.ctx)
        except Exception:
            pass

    # ---------------------------------------------------------------- marshalling
    @staticmethod
    def _kf_key(kfs):
        return tuple((k.depth.data_ptr(), k.offset.data_ptr(), k.rgb.data_ptr(), k.logit.data_ptr(),
                      k.scale.data_ptr(), id(k.cam), bool(k.learnable),
                      k.world_transform.data_ptr() if k.world_transform is not None else 0) for k in kfs)

    def kf_structs(self, kfs: Sequence[DeviceKeyframe]):
        key = ("kf", self._kf_key(kfs))
        hit = self._cache.get(key)
        if hit is None:
            arr = (B.sgad_keyframe * len(kfs))()
            for i, k in enumerate(kfs):
                arr[i] = B.sgad_keyframe(_ptr(k.depth), _ptr(k.offset), _ptr(k.rgb), _ptr(k.logit), _ptr(k.scale),
                                         _cam(k.cam), int(k.learnable), _ptr(k.world_transform))
            if len(self._cache) > 64:
                self._cache.clear()
            self._cache[key] = (arr, list(kfs))        # keep the keyframes (and cameras) alive
            return arr
        return hit[0]

    def view_structs(self, views):
        key = ("views", tuple(id(v) for v in views))
        arr = self._cache.get(key)
        if arr is None:
            if len(self._cache) > 256:
                self._cache.clear()
            arr = (B.sgad_camera * len(views))()
            for i, v in enumerate(views):
                arr[i] = _cam(v)
            self._cache[key] = (arr, list(views))      # keep the camera objects alive
            return arr
        return arr[0]

    @staticmethod
    def stream() -> int:
        return torch.cuda.current_stream().cuda_stream

    @property
    def ws_ptr(self) -> int:
        return self.workspace.data_ptr()

    @property
    def ws_bytes(self) -> int:
        return self.workspace.numel()

    # -------------------------------------------------------------------- calls
    def plan(self, kfs, views, slack: float = 1.15, min_extra: int = 4096) -> int:
        """Size the workspace: counts the keys of these inputs (synchronises) and keeps
        room for `slack` times as many. Returns the key capacity."""
        ka, va = self.kf_structs(kfs), self.view_structs(views)
        base = B.sgad_workspace_size(self.ctx, ka, va, 0)
        if self.workspace is None or self.workspace.numel() < base:
            self.workspace = torch.empty(base, dtype=torch.uint8, device="cuda")
        n = B.sgad_count_keys(self.ctx, ka, va, self.ws_ptr, self.ws_bytes, self.stream())
        cap = int(n * slack) + min_extra
        self.reserve(kfs, views, cap)
        return n

    def _grow(self, nbytes: int) -> None:
        if self.workspace is None or self.workspace.numel() < nbytes:
            self.workspace = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
            self.workspace[:256].zero_()          # device status block starts cleared

    def reserve(self, kfs, views, key_capacity: int) -> None:
        ka, va = self.kf_structs(kfs), self.view_structs(views)
        need = B.sgad_workspace_size(self.ctx, ka, va, key_capacity)
        if self.workspace is None or self.workspace.numel() < need:
            old = self.workspace
            self.workspace = torch.empty(need, dtype=torch.uint8, device="cuda")
            self.workspace[:256].zero_()          # device status block starts cleared
            if old is not None:                   # keep the projection state of plan()
                self.workspace[:old.numel()].copy_(old)
        self.key_capacity = key_capacity

    @staticmethod
    def _images(images):
        out = (B.sgad_images * len(images))()
        for i, im in enumerate(images):
            out[i] = B.sgad_images(_ptr(im["rgb"]), _ptr(im["depth"]), _ptr(im["alpha"]))
        return out

    @staticmethod
    def _grads(grads_in, grads_out):
        gi = (B.sgad_image_grads * len(grads_in))()
        for i, g in enumerate(grads_in):
            gi[i] = B.sgad_image_grads(_ptr(g.get("rgb")), _ptr(g.get("depth")), _ptr(g.get("alpha")),
                                       _ptr(g.get("pose")))
        go = (B.sgad_keyframe_grads * len(grads_out))()
        for i, g in enumerate(grads_out):
            if g is not None:
                go[i] = B.sgad_keyframe_grads(_ptr(g["d_offset"]), _ptr(g["d_rgb"]), _ptr(g["d_logit"]),
                                              _ptr(g["d_scale"]))
        return gi, go

    def forward(self, kfs, views, images) -> None:
        ka, va = self.kf_structs(kfs), self.view_structs(views)
        B.sgad_forward(self.ctx, ka, va, self._images(images), self.ws_ptr, self.ws_bytes, self.key_capacity,
                       self.stream())

    def backward(self, kfs, views, grads_in, grads_out) -> None:
        """grads_in: per view dict of d_rgb / d_depth / d_alpha tensors (missing = 0) and
        optionally "pose", a 12-float tensor that receives d loss / d (world->cam 3x4);
        grads_out: per keyframe dict of d_offset / d_rgb / d_logit / d_scale tensors
        (None for fixed keyframes)."""
        ka, va = self.kf_structs(kfs), self.view_structs(views)
        gi, go = self._grads(grads_in, grads_out)
        B.sgad_backward(self.ctx, ka, va, gi, go, self.ws_ptr, self.ws_bytes, self.key_capacity, self.stream())

    def autotune(self, kfs, views, images, grads_in, grads_out, reps: int = 5, slack: float = 1.15):
        """Runs the library's autotuner on these inputs (synchronous), adopts its choice of
        tile shape, batch sizes and schedules, and re-plans the workspace for that tile
        shape. The workspace is first grown to hold the keys of the largest tile shape.
        Returns the timing rows."""
        ka, va = self.kf_structs(kfs), self.view_structs(views)
        need_bytes = 0
        for shape in B.TILE_SHAPES:            # workspace for the keys of every shape tried
            o = B.sgad_options.from_buffer_copy(self.options)
            o.tile_w, o.tile_h = shape
            c = B.sgad_create(o)
            try:
                base = B.sgad_workspace_size(c, ka, va, 0)
                self._grow(base)
                n = B.sgad_count_keys(c, ka, va, self.ws_ptr, self.ws_bytes, self.stream())
                need_bytes = max(need_bytes, B.sgad_workspace_size(c, ka, va, n))
            finally:
                B.sgad_destroy(c)
        self._grow(need_bytes)
        gi, go = self._grads(grads_in, grads_out)
        rows = B.sgad_autotune(self.ctx, ka, va, self._images(images), gi, go, self.ws_ptr, self.ws_bytes, reps,
                               self.stream())
        self.options = B.sgad_get_options(self.ctx)
        self.plan(kfs, views, slack=slack)
        return rows

    def check(self):
        """(status, n_keys, keys_needed) of the last forward; synchronises."""
        return B.sgad_check(self.ctx, self.ws_ptr, self.ws_bytes, self.stream())

    def stats(self) -> dict:
        s = B.sgad_read_stats(self.ctx, self.ws_ptr, self.ws_bytes, self.stream())
        return dict(n_keys=s.n_keys, keys_needed=s.keys_needed, n_pairs=s.n_pairs, n_evals=s.n_evals,
                    n_sort_exact=s.n_sort_exact)

    def profile(self, enable: bool = True) -> None:
        B.sgad_profile_enable(self.ctx, enable)

    def stage_ms(self) -> dict:
        return dict(zip(B.STAGE_NAMES, B.sgad_profile_read(self.ctx)))

    def state(self, kfs, views):
        """Copies of the forward state: tile offsets (n_tiles + 1), sorted entries,
        per-pixel final transmittance and contributor count (views concatenated)."""
        ka, va = self.kf_structs(kfs), self.view_structs(views)
        sv = B.sgad_state(self.ctx, ka, va, self.ws_ptr, self.ws_bytes, self.key_capacity)
        ws0 = self.ws_ptr
        w = self.workspace

        def view(ptr, n, dtype, itemsize):
            off = ptr - ws0
            return w[off:off + n * itemsize].view(dtype).clone()

        offs = view(sv.tile_offsets, sv.n_tiles + 1, torch.int32, 4)
        n_keys = int(offs[-1].item()) & 0xffffffff
        entries = view(sv.entries, n_keys, torch.int64, 8)
        t_final = view(sv.t_final, sv.n_pixels, torch.float32, 4)
        n_contrib = view(sv.n_contrib, sv.n_pixels, torch.int32, 4)
        return offs, entries, t_final, n_contrib

    def l1_loss_grad(self, views, images, target_rgb, target_depth, rgb_weight, depth_weight, d_rgb, d_depth,
                     loss_accum: Optional[torch.Tensor] = None, valid_count: Optional[torch.Tensor] = None,
                     min_alpha: float = -1.0):
        """Eq. 1's L1 terms and their image gradients; min_alpha >= 0 keeps only pixels whose
        rendered alpha exceeds it (silhouette mask)."""
        va = self.view_structs(views)
        rend = (B.sgad_images * len(views))()
        for i, im in enumerate(images):
            rend[i] = B.sgad_images(_ptr(im["rgb"]), _ptr(im["depth"]), _ptr(im["alpha"]))
        tr = B.ptr_array([_ptr(t) for t in target_rgb])
        td = B.ptr_array([_ptr(t) for t in target_depth]) if target_depth is not None else None
        dr = B.ptr_array([_ptr(t) for t in d_rgb])
        dd = B.ptr_array([_ptr(t) for t in d_depth]) if d_depth is not None else None
        B.sgad_l1_loss_grad(va, rend, tr, td, rgb_weight, depth_weight, dr, dd,
                            _ptr(loss_accum) if loss_accum is not None else None,
                            valid_count.data_ptr() if valid_count is not None else None, self.stream(),
                            min_alpha=min_alpha)

    def ssim_loss_grad(self, views, images, target_rgb, weight, d_rgb, loss_accum: Optional[torch.Tensor] = None):
        """tau L_S of Eq. 1 for every view, ADDED to d_rgb (call after l1_loss_grad)."""
        va = self.view_structs(views)
        need = B.sgad_ssim_workspace_size(va)
        if self._ssim_ws is None or self._ssim_ws.numel() < need:
            self._ssim_ws = torch.empty(max(need, 256), dtype=torch.uint8, device="cuda")
        rend = (B.sgad_images * len(views))()
        for i, im in enumerate(images):
            rend[i] = B.sgad_images(_ptr(im["rgb"]), _ptr(im["depth"]), _ptr(im["alpha"]))
        tr = B.ptr_array([_ptr(t) for t in target_rgb])
        dr = B.ptr_array([_ptr(t) for t in d_rgb])
        B.sgad_ssim_loss_grad(va, rend, tr, weight, dr, _ptr(loss_accum) if loss_accum is not None else None,
                              self._ssim_ws.data_ptr(), self._ssim_ws.numel(), self.stream())


class SplatFn(torch.autograd.Function):
    """Differentiable splat(G, p_k) of Sec. 3.2 over all keyframes and views.

    apply(splatter, keyframes, views, *params) with params = (offset, rgb, logit, scale)
    of every keyframe in order; returns (rgb, depth, alpha) of every view in order. The
    keyframes' `depth` tensors and cameras are taken from `keyframes` (not
    differentiated)."""

    @staticmethod
    def forward(ctx, splatter: Splatter, keyframes, views, *params):
        kfs = []
        for i, k in enumerate(keyframes):
            off, rgb, logit, scale = params[4 * i:4 * i + 4]
            kfs.append(DeviceKeyframe(k.cam, k.depth, off.contiguous(), rgb.contiguous(), logit.contiguous(),
                                      scale.contiguous(), k.learnable))
        images = alloc_images(views)
        splatter.forward(kfs, views, images)
        ctx.splatter, ctx.kfs, ctx.views = splatter, kfs, views
        outs = []
        for im in images:
            outs += [im["rgb"], im["depth"], im["alpha"]]
        return tuple(outs)

    @staticmethod
    def backward(ctx, *grads):
        kfs, views = ctx.kfs, ctx.views
        gin = []
        for i in range(len(views)):
            g = grads[3 * i:3 * i + 3]
            gin.append({k: (t.contiguous() if t is not None else None) for k, t in zip(("rgb", "depth", "alpha"), g)})
        gout = []
        for k in kfs:
            if k.learnable:
                gout.append(dict(d_offset=torch.empty_like(k.offset), d_rgb=torch.empty_like(k.rgb),
                                 d_logit=torch.empty_like(k.logit), d_scale=torch.empty_like(k.scale)))
            else:
                gout.append(None)
        ctx.splatter.backward(kfs, views, gin, gout)
        res = [None, None, None]
        for g in gout:
            if g is None:
                res += [None] * 4
            else:
                res += [g["d_offset"], g["d_rgb"], g["d_logit"], g["d_scale"]]
        return tuple(res)
