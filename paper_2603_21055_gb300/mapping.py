"""Mapping iterations (Sec. 3.2, Eq. 1) on the GPU.

One iteration renders every keyframe of the window into every view (forward splatting),
takes the L1 colour + depth loss gradient against the observed RGB-D (plus the SSIM term
when the scene's ssim_weight is nonzero), runs the adjoint
into offset, colour, opacity logit and scale of the learnable keyframes, and applies one
Adam step with the learning rates of the supplementary Sec. A (colour 0.0025, radius
0.005, opacity 0.05, offset 0.01; the radius rate is applied to log s). All of it is
library launches on one stream; `capture()` records one iteration as a CUDA graph so that
`step()` replays it with a single launch from the host.
"""
from __future__ import annotations

import math
from typing import Optional

import torch

from . import binding as B
from . import splat

LR = dict(offset=0.01, rgb=0.0025, logit=0.05, scale=0.005)
PARAMS = (("offset", "d_offset"), ("rgb", "d_rgb"), ("logit", "d_logit"), ("scale", "d_scale"))


class Mapper:
    """Device state of one keyframe window: parameters, Adam moments, images, gradients,
    targets and the library workspace."""

    def __init__(self, scene, tile=(16, 16), slack: float = 1.3, lr: Optional[dict] = None,
                 freeze_offset: bool = False, kfs=None, work_split: Optional[dict] = None, targets=None,
                 loss: Optional[torch.Tensor] = None, options=None):
        """kfs, targets ((rgb list, depth list)) and loss (one float) may be given as device
        tensors (e.g. the views of splat.upload_window); options: a complete sgad_options
        used instead of tile, freeze_offset and work_split."""
        self.scene = scene
        self.views = scene.views
        self.lr = dict(LR, **(lr or {}))
        if options is not None:
            self.sp = splat.Splatter(options=options)
            freeze_offset = bool(options.freeze_offset)
        else:
            self.sp = splat.Splatter(tile=tile, freeze_offset=freeze_offset, **(work_split or {}))
        self.kfs = kfs if kfs is not None else splat.upload_keyframes(scene)
        self.trgb, self.tdep = targets if targets is not None else splat.upload_targets(scene)
        self.images = splat.alloc_images(self.views)
        self.d_rgb = [torch.empty_like(im["rgb"]) for im in self.images]
        self.d_dep = [torch.empty_like(im["depth"]) for im in self.images]
        self.gin = [dict(rgb=r, depth=d) for r, d in zip(self.d_rgb, self.d_dep)]
        self.loss = loss if loss is not None else torch.zeros(1, device="cuda")
        self.valid = torch.zeros(len(self.views), dtype=torch.int32, device="cuda")
        self.grads = [dict(d_offset=torch.empty_like(k.offset), d_rgb=torch.empty_like(k.rgb),
                           d_logit=torch.empty_like(k.logit), d_scale=torch.empty_like(k.scale))
                      if k.learnable else None for k in self.kfs]
        self.moments = [{n: (torch.zeros_like(getattr(k, n)), torch.zeros_like(getattr(k, n))) for n, _ in PARAMS}
                        if k.learnable else None for k in self.kfs]
        self.step_counter = torch.zeros(1, dtype=torch.int32, device="cuda")
        tensors = []
        for k, g, mo in zip(self.kfs, self.grads, self.moments):
            if g is None:
                continue
            for n, gn in PARAMS:
                if n == "offset" and freeze_offset:
                    continue
                p = getattr(k, n)
                m, v = mo[n]
                mode = B.SGAD_ADAM_LOG if n == "scale" else B.SGAD_ADAM_PLAIN
                tensors.append(B.sgad_adam_tensor(p.data_ptr(), g[gn].data_ptr(), m.data_ptr(), v.data_ptr(),
                                                  p.numel(), self.lr[n], mode))
        self.adam = (B.sgad_adam_tensor * max(1, len(tensors)))(*tensors)
        self.n_adam = len(tensors)
        self.graph: Optional[torch.cuda.CUDAGraph] = None
        self.n_keys = self.sp.plan(self.kfs, self.views, slack=slack)

    # ------------------------------------------------------------------ one step
    def forward(self):
        self.sp.forward(self.kfs, self.views, self.images)

    def step_eager(self):
        self._step(range(len(self.views)))

    def step_views(self, idx):
        """One iteration that renders, and takes the loss of, only the views `idx` (indices
        into the scene's views); the workspace planned for all views serves any subset."""
        self._step(list(idx))

    def _step(self, idx):
        sp = self.sp
        pick = lambda xs: [xs[k] for k in idx]
        views, images, d_rgb = pick(self.views), pick(self.images), pick(self.d_rgb)
        sp.forward(self.kfs, views, images)
        self.loss.zero_()
        sp.l1_loss_grad(views, images, pick(self.trgb), pick(self.tdep), self.scene.rgb_weight,
                        self.scene.depth_weight, d_rgb, pick(self.d_dep), self.loss, self.valid)
        if self.scene.ssim_weight != 0:
            sp.ssim_loss_grad(views, images, pick(self.trgb), self.scene.ssim_weight, d_rgb, self.loss)
        sp.backward(self.kfs, views, pick(self.gin), self.grads)
        if self.n_adam:
            B.sgad_adam_step_multi(self.adam, 0.9, 0.999, 1e-15, self.step_counter.data_ptr(), sp.stream())

    def eval_loss(self):
        """Render every view and put the mapping loss of Eq. 1 (the scene's weights) into
        self.loss, on the device: no gradient step, no host synchronisation."""
        sp = self.sp
        sp.forward(self.kfs, self.views, self.images)
        self.loss.zero_()
        sp.l1_loss_grad(self.views, self.images, self.trgb, self.tdep, self.scene.rgb_weight,
                        self.scene.depth_weight, self.d_rgb, self.d_dep, self.loss, self.valid)
        if self.scene.ssim_weight != 0:
            sp.ssim_loss_grad(self.views, self.images, self.trgb, self.scene.ssim_weight, self.d_rgb, self.loss)

    def capture(self):
        """Record one iteration as a CUDA graph (after one eager warm-up on a side stream)."""
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self.step_eager()
        torch.cuda.current_stream().wait_stream(s)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.step_eager()
        self.graph = g

    def step(self):
        if self.graph is not None:
            self.graph.replay()
        else:
            self.step_eager()

    def launches_per_step(self) -> int:
        """Library kernels per iteration: projection+count, scan, emission, sort, forward
        compositing (one launch per view with the per-view schedule); valid-depth count and
        L1 gradient; the two SSIM passes when that term is on; backward compositing,
        finalisation; multi-tensor Adam and its step counter."""
        o = self.sp.options
        per = lambda sched: len(self.views) if sched == B.SGAD_SCHEDULE_PER_VIEW else 1
        n = 4 + per(o.fwd_schedule) + (2 if self.scene.depth_weight != 0 else 1) + per(o.bwd_schedule) + 1
        n += 2 if self.scene.ssim_weight != 0 else 0
        return n + (2 if self.n_adam else 0)

    def autotune(self, reps: int = 5):
        """Let the library's autotuner pick tile shape, batch sizes and schedules for this
        window (on the current gradients of one eager iteration); drops a captured graph."""
        self.step_eager()
        rows = self.sp.autotune(self.kfs, self.views, self.images, self.gin, self.grads, reps=reps)
        self.graph = None
        return rows

    # ------------------------------------------------------------------ checks
    def ensure_capacity(self, slack: float = 1.3) -> bool:
        """False (and a bigger workspace, which invalidates a captured graph) if any
        forward since the last check ran out of key slots."""
        s, _, need = self.sp.check()
        if s != 0:
            self.sp.reserve(self.kfs, self.views, int(need * slack) + 4096)
            self.graph = None
            return False
        return True

    def psnr(self) -> float:
        """Mean PSNR over the views of the last forward: 10 log10(1 / MSE), RGB in [0, 1]."""
        vals = []
        for im, t in zip(self.images, self.trgb):
            mse = torch.mean((im["rgb"].clamp(0, 1) - t) ** 2).item()
            vals.append(10.0 * math.log10(1.0 / max(mse, 1e-12)))
        return sum(vals) / len(vals)


class StreamedWindows:
    """Mapping iterations on a window held in pinned host memory: every iteration uploads
    the window (keyframe planes, targets, loss slot: one copy, the layout of
    splat.upload_window) and reads the updated parameters and the loss back (one copy).
    Two device copies of the window alternate, so that one iteration's copies run on a
    copy stream while the other copy's iteration runs; `replay()` runs two iterations (A,
    then B) as one CUDA graph:
        copy stream:    read back B (previous)  upload B  | read back A  upload A (next)
        compute stream: iteration A                       | iteration B
    Every iteration's upload precedes it and its read-back follows it; `finish()` reads
    back the last B. `host_in` holds the window every iteration starts from;
    `host_out[0]`, `host_out[1]` the state after the last A and B iterations."""

    def __init__(self, scene, options=None, slack: float = 1.3):
        self.windows = []
        for _ in range(2):
            buf, n_state, kfs, trgb, tdep, loss = splat.upload_window(scene)
            m = Mapper(scene, kfs=kfs, targets=(trgb, tdep), loss=loss, options=options, slack=slack)
            self.windows.append((buf, m))
        self.n_state = n_state
        self.host_in = self.windows[0][0].cpu().pin_memory()
        self.host_out = [torch.empty(n_state, dtype=torch.float32, pin_memory=True) for _ in range(2)]
        self.copy_stream = torch.cuda.Stream()
        self.graph: Optional[torch.cuda.CUDAGraph] = None

    @property
    def mappers(self):
        return [m for _, m in self.windows]

    def ensure_capacity(self, tries: int = 3) -> bool:
        """Eager iterations on both copies until their key capacity suffices (from the
        current device contents); drops a captured graph."""
        ok = True
        for buf, m in self.windows:
            for _ in range(tries):
                m.step_eager()
                torch.cuda.synchronize()
                if m.ensure_capacity():
                    break
            ok = ok and m.ensure_capacity()
        self.graph = None
        return ok

    def _pair(self):
        (buf_a, m_a), (buf_b, m_b) = self.windows
        n, cs = self.n_state, self.copy_stream
        main = torch.cuda.current_stream()
        cs.wait_stream(main)
        with torch.cuda.stream(cs):
            self.host_out[1].copy_(buf_b[:n], non_blocking=True)     # the previous iteration B's result
            buf_b.copy_(self.host_in, non_blocking=True)             # this iteration B's inputs
        in_b = torch.cuda.Event()
        in_b.record(cs)
        m_a.step_eager()                                             # iteration A (inputs uploaded before)
        done_a = torch.cuda.Event()
        done_a.record(main)
        with torch.cuda.stream(cs):
            cs.wait_event(done_a)
            self.host_out[0].copy_(buf_a[:n], non_blocking=True)     # iteration A's result
            buf_a.copy_(self.host_in, non_blocking=True)             # the next iteration A's inputs
        main.wait_event(in_b)
        m_b.step_eager()                                             # iteration B
        main.wait_stream(cs)

    def capture(self):
        """Upload A's first inputs, run one pair eagerly on a side stream, then record the
        pair as a CUDA graph."""
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self.windows[0][0].copy_(self.host_in, non_blocking=True)
            self._pair()
        torch.cuda.current_stream().wait_stream(s)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self._pair()
        self.graph = g

    def replay(self):
        """Two iterations (A and B) with their copies."""
        if self.graph is None:
            self.capture()
        self.graph.replay()

    def finish(self):
        """Read back the last iteration B's result (on the current stream)."""
        buf_b = self.windows[1][0]
        self.host_out[1].copy_(buf_b[:self.n_state], non_blocking=True)
