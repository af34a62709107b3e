"""Learned initialisation of new keyframes: data, targets from the plain mapping, training
of the proposal net, and the seconds-to-PSNR comparison against the zero initialisation.

Protocol (readings of the workload; the paper has no learned part):
  * A room is a seeded box room (synth.make_room) seen from `frames_per_room` frames on a
    smooth path (~10 cm / ~5 degrees apart), 640x480, fx = fy = 600. Each frame has the
    ray-cast colour and depth; the observed depth adds N(0, 1 cm) noise and is quantised
    to 2 mm.
  * A mapping window is 5 consecutive frames. Every frame of the window is a learnable
    keyframe (pixel-aligned Gaussians at the observed depth, colour = observed colour,
    radius D / f as in Supp. A); the window is fitted against 4 neighbour views, the
    poses halfway between consecutive frames of the window (rotation by half the
    relative angle, translation averaged), whose ray-cast colour and observed depth are
    the targets, so that no view ray passes through a Gaussian by construction. The loss
    is Eq. 1 without the SSIM term, rho = 0.8 (colour) and sigma = 1.0 (depth), with the
    Supp. A learning rates.
  * The plain initialisation is delta = 0 and opacity logit 0 (opacity 0.5).
  * Targets: delta and logit of every keyframe after 100 plain mapping iterations.
  * The learned arm keeps the plain zero-offset initialisation as fallback and as the check
    on the net's error: after inference it renders the window with the prediction, with zero
    offsets and the predicted opacities, and with the plain initialisation, and maps from
    the one with the lowest Eq. 1 loss.
  * Evaluation on held-out rooms: wall time (CUDA events) from the window's arrival on the
    GPU, including the net's inference and the fallback check for the learned arm, until
    the mean PSNR over the window's views (RGB clamped to [0, 1]) first reaches a target;
    and the per-pixel |delta_pred - delta_plain| against the plain run's converged
    offsets.
"""
from __future__ import annotations

import math
import multiprocessing as mp_
import time
from typing import Dict, List, Optional

import numpy as np

from . import synth

FRAME = (640, 480, 600.0, 320.0, 240.0)
DEPTH_NOISE = 0.01
DEPTH_QUANT = 0.002
PLAIN_LOGIT = 0.0
WINDOW = 5
RGB_WEIGHT, DEPTH_WEIGHT = 0.8, 1.0
TARGET_DB = 30.0


def midpoint_pose(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """cam->world pose halfway between two poses: the rotation turned by half the
    relative angle about its axis, the mean of the positions."""
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    rel = a[:, :3].T @ b[:, :3]
    ang = math.acos(float(np.clip((np.trace(rel) - 1.0) / 2.0, -1.0, 1.0)))
    r = a[:, :3]
    if ang > 1e-9:
        axis = np.array([rel[2, 1] - rel[1, 2], rel[0, 2] - rel[2, 0], rel[1, 0] - rel[0, 1]]) / (2.0 * math.sin(ang))
        r = r @ synth.rotation_about(axis, 0.5 * ang)
    return np.concatenate([r, (0.5 * (a[:, 3] + b[:, 3]))[:, None]], axis=1)


def room_frames(seed: int, n_frames: int = 40, size=FRAME) -> Dict[str, np.ndarray]:
    """Frames of one seeded room: cam->world poses, colour, ray-cast and observed depth;
    and the same at the n_frames - 1 poses halfway between consecutive frames (the
    neighbour views)."""
    rng = np.random.default_rng(seed)
    centre = np.array([3.0, 2.5, 1.5])
    room = synth.make_room(rng, keep_free=(centre, 1.1))
    poses = synth.keyframe_path(rng, n_frames, centre)
    mids = [midpoint_pose(poses[i], poses[i + 1]) for i in range(n_frames - 1)]
    w, h, f, cx, cy = size
    out = dict(seed=seed, size=np.asarray(size, np.float64))
    for tag, ps in (("", poses), ("mid_", mids)):
        n = len(ps)
        rgb = np.empty((n, 3, h, w), np.float32)
        depth = np.empty((n, h, w), np.float32)
        for i, p in enumerate(ps):
            depth[i], rgb[i] = synth.raycast(room, p, w, h, f, f, cx, cy)
        noisy = depth + rng.normal(0.0, DEPTH_NOISE, size=depth.shape)
        obs = (np.round(noisy / DEPTH_QUANT) * DEPTH_QUANT).astype(np.float32)
        out.update({tag + "poses": np.stack([synth._f32pose(p) for p in ps]), tag + "rgb": rgb,
                    tag + "depth": depth, tag + "obs": obs})
    return out


def window_scene(fr, idx, offsets=None, logits=None) -> synth.Scene:
    """Scene of the consecutive frames `idx` of one room: each frame a learnable keyframe
    (plain initialisation unless offsets / logits are given), fitted against the
    neighbour views halfway between consecutive frames of the window."""
    w, h, f, cx, cy = fr["size"]
    w, h = int(w), int(h)
    kfs, views, trgb, tdep = [], [], [], []
    for j, i in enumerate(idx):
        obs = fr["obs"][i]
        off = np.zeros_like(obs) if offsets is None else np.asarray(offsets[j], np.float32)
        lg = np.full_like(obs, PLAIN_LOGIT) if logits is None else np.asarray(logits[j], np.float32)
        kfs.append(synth.Keyframe(synth.Camera(w, h, f, f, cx, cy, fr["poses"][i]), obs, off, fr["rgb"][i], lg,
                                  (obs / np.float32(f)).astype(np.float32), True))
    for i in idx[:-1]:
        c2w = fr["mid_poses"][i].astype(np.float64)
        views.append(synth.Camera(w, h, f, f, cx, cy, synth._f32pose(synth.pose_inverse(c2w))))
        trgb.append(fr["mid_rgb"][i])
        tdep.append(fr["mid_obs"][i])
    return synth.Scene(kfs, views, trgb, tdep, DEPTH_WEIGHT, RGB_WEIGHT, "window%d" % fr["seed"])


def windows(n_frames: int):
    return [list(range(s, s + WINDOW)) for s in range(0, n_frames - WINDOW + 1, WINDOW)]


def _gen(args):
    seed, n_frames, size = args
    return room_frames(seed, n_frames, size)


def generate_rooms(seeds, n_frames: int, workers: int, size=FRAME):
    """Yields room_frames(seed) for each seed, in order, computed by a spawn-context pool
    (safe next to CUDA in the calling process)."""
    ctx = mp_.get_context("spawn")
    with ctx.Pool(workers) as pool:
        for fr in pool.imap(_gen, [(s, n_frames, tuple(size)) for s in seeds]):
            yield fr


# ------------------------------------------------------------------ GPU parts

def mean_psnr_into(mapper, out) -> None:
    """out[0] = mean over views of 10 log10(1 / MSE) of the last render (device ops)."""
    import torch
    vals = []
    for im, t in zip(mapper.images, mapper.trgb):
        mse = torch.mean((im["rgb"].clamp(0.0, 1.0) - t) ** 2).clamp_min(1e-12)
        vals.append(-10.0 * torch.log10(mse))
    out.copy_(torch.stack(vals).mean().reshape(1))


def plain_targets(fr, idx, iters: int = 100):
    """(offsets, logits) of the window's keyframes after `iters` plain mapping iterations."""
    from .mapping import Mapper
    mp = Mapper(window_scene(fr, idx))
    for _ in range(iters):
        mp.step_eager()
    if not mp.ensure_capacity():            # rerun with room for every key
        mp = Mapper(window_scene(fr, idx))
        for _ in range(iters):
            mp.step_eager()
        assert mp.ensure_capacity()
    return [k.offset.clone() for k in mp.kfs], [k.logit.clone() for k in mp.kfs]


def learned_init(mp, net, rgb_b, dep_b, off_b, lg_b, plain):
    """Learned initialisation with the plain zero-offset one as fallback and check: runs the
    net on the window's RGB-D (rgb_b (n, 3, H, W), dep_b (n, H, W)) into off_b / lg_b, then
    renders the window with three initialisations, in this order of preference: the
    prediction; zero offsets with the predicted opacities; and the plain initialisation the
    keyframes hold (`plain`: their (offset, logit) pairs). The one with the lowest Eq. 1
    loss stays in the keyframes (ties go to the earlier one). Device operations only, no
    host synchronisation; returns a device int32 tensor: 0, 1 or 2, the one kept."""
    import torch
    net.forward(rgb_b, dep_b, off_b, lg_b)
    mp.eval_loss()
    losses = [None, None, mp.loss.clone()]              # plain
    for j, k in enumerate(mp.kfs):
        k.logit.copy_(lg_b[j])
    mp.eval_loss()
    losses[1] = mp.loss.clone()                         # zero offsets, predicted opacity
    for j, k in enumerate(mp.kfs):
        k.offset.copy_(off_b[j])
    mp.eval_loss()
    losses[0] = mp.loss.clone()                         # prediction
    l = torch.cat(losses)
    pick = torch.argmin(l).to(torch.int32).reshape(1)   # first minimum on ties
    use_off = pick == 0
    use_lg = pick <= 1
    for k, (o, lg0) in zip(mp.kfs, plain):
        torch.where(use_off, k.offset, o, out=k.offset)
        torch.where(use_lg, k.logit, lg0, out=k.logit)
    return pick


def time_to_psnr(fr, idx, net=None, iters: int = 100, target_db: float = TARGET_DB):
    """One arm of the comparison on one window. The window's keyframes and targets are
    uploaded first (their arrival); the clock starts there. The learned arm (net given)
    runs learned_init (net inference, then the best of the prediction, zero offsets with
    the predicted opacities and the plain initialisation by first-render loss); both arms
    then run mapping iterations (each one CUDA graph replay), recording the mean PSNR of
    every render. Returns a dict with the seconds to target (None if not reached), PSNR and
    time per iteration, final offsets, the prediction and which initialisation the learned
    arm kept (0 prediction, 1 zero offsets + predicted opacities, 2 plain)."""
    import torch
    from .mapping import Mapper
    mp = Mapper(window_scene(fr, idx))
    init = [(k.offset.clone(), k.logit.clone()) for k in mp.kfs]
    mp.capture()                          # warm-up iteration + capture; state reset below
    n = len(idx)
    h, w = mp.kfs[0].depth.shape
    off_b = torch.empty(n, h, w, device="cuda")
    lg_b = torch.empty(n, h, w, device="cuda")

    def reset():
        for k, (o, l) in zip(mp.kfs, init):
            k.offset.copy_(o)
            k.logit.copy_(l)
        for mo in mp.moments:
            for m, v in mo.values():
                m.zero_()
                v.zero_()
        mp.step_counter.zero_()
        with torch.no_grad():
            for k, kf in zip(mp.kfs, mp.scene.keyframes):
                k.rgb.copy_(torch.as_tensor(kf.rgb).cuda())
                k.scale.copy_(torch.as_tensor(kf.scale).cuda())

    reset()
    rgb_b = torch.stack([k.rgb for k in mp.kfs]).contiguous()      # observed colour and depth
    dep_b = torch.stack([k.depth for k in mp.kfs]).contiguous()
    if net is not None:                   # warm the net's kernels once outside the timing
        net.forward(rgb_b, dep_b, off_b, lg_b)
    hist = torch.zeros(iters, device="cuda")
    cur = torch.zeros(1, device="cuda")
    ev0 = torch.cuda.Event(enable_timing=True)
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(iters)]
    torch.cuda.synchronize()
    ev0.record()
    kept = learned_init(mp, net, rgb_b, dep_b, off_b, lg_b, init) if net is not None else None
    for i in range(iters):
        mp.graph.replay()
        mean_psnr_into(mp, cur)
        hist[i:i + 1].copy_(cur)
        evs[i].record()
    torch.cuda.synchronize()
    ok = mp.ensure_capacity()
    h_ = hist.cpu().numpy()
    t_ = np.array([ev0.elapsed_time(e) / 1e3 for e in evs])
    secs, its = seconds_to(h_, t_, target_db)
    return dict(seconds=secs, psnr=h_, times=t_, offsets=[k.offset.clone() for k in mp.kfs], capacity_ok=ok,
                iters_to_target=its, predicted=[off_b[j].clone() for j in range(n)] if net is not None else None,
                kept=int(kept.item()) if kept is not None else None)


def seconds_to(psnr, times, target_db):
    """(seconds, iterations) until the first render with PSNR >= target_db, or
    (None, None) if none reached it."""
    hit = np.nonzero(np.asarray(psnr) >= target_db)[0]
    if not len(hit):
        return None, None
    return float(times[int(hit[0])]), int(hit[0]) + 1


class Dataset:
    """Training frames and targets resident on the GPU."""

    def __init__(self, capacity: int, size=FRAME):
        import torch
        w, h = int(size[0]), int(size[1])
        self.rgb = torch.empty(capacity, 3, h, w, device="cuda")
        self.obs = torch.empty(capacity, h, w, device="cuda")
        self.td = torch.empty(capacity, h, w, device="cuda")
        self.tl = torch.empty(capacity, h, w, device="cuda")
        self.n = 0

    def add(self, rgb, obs, offsets, logits) -> None:
        import torch
        i = self.n
        self.rgb[i].copy_(torch.as_tensor(rgb))
        self.obs[i].copy_(torch.as_tensor(obs))
        self.td[i].copy_(offsets)
        self.tl[i].copy_(logits)
        self.n += 1


def build_dataset(seeds, frames_per_room: int, workers: int, log=print, size=FRAME) -> Dataset:
    ds = Dataset(len(seeds) * (frames_per_room // WINDOW) * WINDOW, size)
    t0 = time.perf_counter()
    for r, fr in enumerate(generate_rooms(seeds, frames_per_room, workers, size)):
        for idx in windows(frames_per_room):
            offs, lgs = plain_targets(fr, idx)
            for j, i in enumerate(idx):
                ds.add(fr["rgb"][i], fr["obs"][i], offs[j], lgs[j])
        if log and (r + 1) % 5 == 0:
            log("rooms %d/%d, frames %d, %.0f s" % (r + 1, len(seeds), ds.n, time.perf_counter() - t0))
    return ds


def train(net, ds: Dataset, steps: int, batch: int = 8, lr: float = 2e-3, seed: int = 0, log=print):
    """Adam on random batches of frames; cosine learning-rate decay. Returns the loss curve
    (every 50 steps)."""
    import torch
    g = torch.Generator(device="cpu").manual_seed(seed)
    curve = []
    h, w = ds.obs.shape[1:]
    rb = torch.empty(batch, 3, h, w, device="cuda")
    ob = torch.empty(batch, h, w, device="cuda")
    tdb = torch.empty(batch, h, w, device="cuda")
    tlb = torch.empty(batch, h, w, device="cuda")
    for s in range(steps):
        idx = torch.randint(0, ds.n, (batch,), generator=g).cuda()
        torch.index_select(ds.rgb, 0, idx, out=rb)
        torch.index_select(ds.obs, 0, idx, out=ob)
        torch.index_select(ds.td, 0, idx, out=tdb)
        torch.index_select(ds.tl, 0, idx, out=tlb)
        net.lr = lr * 0.5 * (1.0 + math.cos(math.pi * s / steps))
        net.train_step(rb, ob, tdb, tlb)
        if s % 50 == 0 or s == steps - 1:
            curve.append((s, float(net.loss.item())))
            if log and s % 500 == 0:
                log("step %d loss %.4f" % (s, curve[-1][1]))
    return curve
