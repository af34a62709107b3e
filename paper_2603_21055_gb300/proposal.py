"""The learned proposal net on the GPU: parameters, training step and inference.

Torch holds the device memory; every step (input packing, the four tensor-core
convolutions, the loss, the adjoint and the Adam update) is a library launch
(include/sgad_net.h, include/sgad.h).
"""
from __future__ import annotations

from typing import Optional

import numpy as np
import torch

from . import binding as B

LAYERS = 4


def padded_shapes():
    return [B.sgad_net_layer_shape(l) for l in range(LAYERS)]


def he_init(seed: int = 0):
    """Seeded He-normal weights (3, 3, cin, cout) and zero biases, float32."""
    rng = np.random.default_rng(seed)
    out = []
    for cin, cout, _, _ in padded_shapes():
        w = rng.normal(0.0, np.sqrt(2.0 / (9 * cin)), size=(3, 3, cin, cout)).astype(np.float32)
        out.append((w, np.zeros(cout, np.float32)))
    return out


class ProposalNet:
    """FP32 master parameters in the library's padded layout, their gradients and Adam
    moments, and one workspace for batches of up to `max_frames` frames of h x w."""

    def __init__(self, params=None, seed: int = 0, device: str = "cuda"):
        params = params if params is not None else he_init(seed)
        self.shapes = padded_shapes()
        self.w, self.b = [], []
        for (wr, br), (cin, cout, cin_p, cout_p) in zip(params, self.shapes):
            wp = np.zeros((9, cin_p, cout_p), np.float32)
            wp[:, :cin, :cout] = np.asarray(wr, np.float32).reshape(9, cin, cout)
            bp = np.zeros(cout_p, np.float32)
            bp[:cout] = br
            self.w.append(torch.as_tensor(wp).to(device))
            self.b.append(torch.as_tensor(bp).to(device))
        self.dw = [torch.zeros_like(t) for t in self.w]
        self.db = [torch.zeros_like(t) for t in self.b]
        self.m = [torch.zeros_like(t) for t in self.w + self.b]
        self.v = [torch.zeros_like(t) for t in self.w + self.b]
        self.step_counter = torch.zeros(1, dtype=torch.int32, device=device)
        self.loss = torch.zeros(1, device=device)
        self.workspace: Optional[torch.Tensor] = None
        self.shape = None
        self._params = B.sgad_net_params()
        self._grads = B.sgad_net_grads()
        for l in range(LAYERS):
            self._params.w[l] = self.w[l].data_ptr()
            self._params.b[l] = self.b[l].data_ptr()
            self._grads.dw[l] = self.dw[l].data_ptr()
            self._grads.db[l] = self.db[l].data_ptr()
        self.lr = 1e-3
        self._adam = None

    # --------------------------------------------------------------- plumbing
    @staticmethod
    def stream() -> int:
        return torch.cuda.current_stream().cuda_stream

    def reserve(self, n: int, h: int, w: int) -> None:
        need = B.sgad_net_workspace_size(n, h, w)
        if self.workspace is None or self.workspace.numel() < need:
            self.workspace = torch.empty(need, dtype=torch.uint8, device="cuda")
            self.workspace[:256].zero_()          # device status word starts cleared
        self.shape = (n, h, w)

    def real_params(self):
        """[(w (3,3,cin,cout), b (cout,))] as float32 numpy arrays (unpadded)."""
        out = []
        for wt, bt, (cin, cout, _, _) in zip(self.w, self.b, self.shapes):
            w = wt.cpu().numpy()[:, :cin, :cout].reshape(3, 3, cin, cout)
            out.append((w, bt.cpu().numpy()[:cout]))
        return out

    # ----------------------------------------------------------------- calls
    def forward(self, rgb: torch.Tensor, depth: torch.Tensor, delta: Optional[torch.Tensor] = None,
                logit: Optional[torch.Tensor] = None) -> None:
        """rgb (N,3,H,W), depth (N,H,W) -> delta (N,H,W) metres and logit (N,H,W)."""
        n, _, h, w = rgb.shape
        self.reserve(n, h, w)
        B.sgad_net_forward(self._params, n, h, w, rgb.data_ptr(), depth.data_ptr(),
                           delta.data_ptr() if delta is not None else 0,
                           logit.data_ptr() if logit is not None else 0, self.workspace.data_ptr(),
                           self.workspace.numel(), self.stream())

    def loss_grad(self, target_delta: torch.Tensor, target_logit: torch.Tensor, logit_weight: float = 1.0,
                  accumulate: bool = False) -> None:
        n, h, w = self.shape
        if not accumulate:
            self.loss.zero_()
        B.sgad_net_loss_grad(n, h, w, target_delta.data_ptr(), target_logit.data_ptr(), logit_weight,
                             self.loss.data_ptr(), self.workspace.data_ptr(), self.workspace.numel(), self.stream())

    def backward(self) -> None:
        n, h, w = self.shape
        B.sgad_net_backward(self._params, self._grads, n, h, w, self.workspace.data_ptr(), self.workspace.numel(),
                            self.stream())

    def adam_step(self, lr: Optional[float] = None) -> None:
        lr = self.lr if lr is None else lr
        if self._adam is None or self._adam[1] != lr:
            ts = []
            for p, g, m, v in zip(self.w + self.b, self.dw + self.db, self.m, self.v):
                ts.append(B.sgad_adam_tensor(p.data_ptr(), g.data_ptr(), m.data_ptr(), v.data_ptr(), p.numel(),
                                             lr, B.SGAD_ADAM_PLAIN))
            self._adam = ((B.sgad_adam_tensor * len(ts))(*ts), lr)
        B.sgad_adam_step_multi(self._adam[0], 0.9, 0.999, 1e-8, self.step_counter.data_ptr(), self.stream())

    def train_step(self, rgb, depth, target_delta, target_logit, logit_weight: float = 1.0) -> None:
        self.forward(rgb, depth)
        self.loss_grad(target_delta, target_logit, logit_weight)
        self.backward()
        self.adam_step()

    def check(self) -> int:
        return B.sgad_net_check(self.workspace.data_ptr(), self.workspace.numel(), self.stream())

    def buffers(self):
        n, h, w = self.shape
        return B.sgad_net_buffers_view(n, h, w, self.workspace.data_ptr(), self.workspace.numel())

    def workspace_array(self, ptr: int, count: int, dtype=torch.bfloat16) -> torch.Tensor:
        """A copy of `count` elements at device address `ptr` inside the workspace."""
        off = int(ptr) - self.workspace.data_ptr()
        size = torch.tensor([], dtype=dtype).element_size()
        return self.workspace[off:off + count * size].view(dtype).clone()

