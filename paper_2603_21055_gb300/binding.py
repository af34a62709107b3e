"""ctypes binding of the C ABI in include/sgad.h (libsgad.so).

Argument marshalling only: every step of the splatting path runs in the CUDA library.
Importing this module loads libsgad.so (building it with nvcc first if it is missing or
stale) and raises if that fails; there is no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os

from . import build as _build

SGAD_OK = 0
SGAD_ERR_INVALID_ARG = -1
SGAD_ERR_CUDA = -2
SGAD_ERR_WORKSPACE_TOO_SMALL = -3
SGAD_ERR_KEY_OVERFLOW = -4
SGAD_ERR_TIMEOUT = -5
SGAD_ERR_UNSUPPORTED = -6
SGAD_ERR_NO_FORWARD = -7
SGAD_MAX_KEYFRAMES = 32
SGAD_MAX_VIEWS = 64

EXPORTS = ["sgad_default_options", "sgad_create", "sgad_destroy", "sgad_last_error", "sgad_workspace_size",
           "sgad_count_keys", "sgad_forward", "sgad_backward", "sgad_check", "sgad_state", "sgad_read_stats",
           "sgad_profile_enable", "sgad_profile_read", "sgad_l1_loss_grad", "sgad_pose_adam_step", "sgad_adam_step",
           "sgad_adam_step_multi", "sgad_forward_noalloc", "sgad_autotune", "sgad_get_options",
           "sgad_ssim_workspace_size", "sgad_ssim_loss_grad", "sgad_fma_burn",
           # include/sgad_gicp.h
           "sgad_gicp_default_params", "sgad_gicp_workspace_size", "sgad_gicp_frame", "sgad_gicp_index",
           "sgad_gicp_correspond", "sgad_gicp_linearize", "sgad_gicp_set_pose", "sgad_gicp_track",
           "sgad_gicp_insert", "sgad_gicp_result",
           # include/sgad_net.h
           "sgad_net_layer_shape", "sgad_net_workspace_size", "sgad_net_forward", "sgad_net_loss_grad",
           "sgad_net_backward", "sgad_net_check", "sgad_net_buffers_view"]
SGAD_NUM_STAGES = 6
STAGE_NAMES = ["binning", "emit", "sort", "composite_fwd", "composite_bwd", "finalize"]


class SgadError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("sgad status %d: %s" % (status, message))
        self.status = status


class sgad_camera(C.Structure):
    _fields_ = [("width", C.c_int32), ("height", C.c_int32), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("pose", C.c_float * 12)]


class sgad_keyframe(C.Structure):
    _fields_ = [("depth", C.c_void_p), ("offset", C.c_void_p), ("rgb", C.c_void_p),
                ("opacity_logit", C.c_void_p), ("scale", C.c_void_p), ("cam", sgad_camera),
                ("learnable", C.c_int32), ("world_transform", C.c_void_p)]


class sgad_images(C.Structure):
    _fields_ = [("rgb", C.c_void_p), ("depth", C.c_void_p), ("alpha", C.c_void_p)]


class sgad_image_grads(C.Structure):
    _fields_ = [("d_rgb", C.c_void_p), ("d_depth", C.c_void_p), ("d_alpha", C.c_void_p), ("d_pose", C.c_void_p)]


class sgad_gicp_params(C.Structure):
    _fields_ = [("stride", C.c_int32), ("k_cov", C.c_int32), ("k_match", C.c_int32), ("max_iters", C.c_int32),
                ("r_max", C.c_float), ("d_overlap", C.c_float), ("tol", C.c_float), ("eps", C.c_float),
                ("src_capacity", C.c_int32), ("map_capacity", C.c_int32)]


class sgad_gaussian_set(C.Structure):
    _fields_ = [("pos", C.c_void_p), ("cov", C.c_void_p), ("normal", C.c_void_p), ("count", C.c_void_p),
                ("capacity", C.c_int32)]


class sgad_gicp_stats(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("converged", C.c_int32), ("n_matches", C.c_int32),
                ("status", C.c_int32), ("cost", C.c_double), ("step", C.c_double)]


class sgad_keyframe_grads(C.Structure):
    _fields_ = [("d_offset", C.c_void_p), ("d_rgb", C.c_void_p), ("d_opacity_logit", C.c_void_p),
                ("d_scale", C.c_void_p)]


SGAD_SCHEDULE_TILES = 0
SGAD_SCHEDULE_PERSISTENT = 1
SGAD_SCHEDULE_PER_VIEW = 2
SCHEDULE_NAMES = {0: "tiles", 1: "persistent", 2: "per_view"}
BATCH_SIZES = (128, 192, 256, 384, 512)          # both compositing passes
FWD_BATCH_SIZES = BATCH_SIZES + (768, 1024)      # forward only
TILE_SHAPES = ((16, 16), (8, 32), (32, 8))


class sgad_options(C.Structure):
    _fields_ = [("tile_w", C.c_int32), ("tile_h", C.c_int32), ("bg", C.c_float * 3),
                ("sort_smem_cap", C.c_int32), ("freeze_offset", C.c_int32), ("fwd_batch", C.c_int32),
                ("bwd_batch", C.c_int32), ("fwd_schedule", C.c_int32), ("bwd_schedule", C.c_int32),
                ("bwd_algorithm", C.c_int32), ("max_blocks", C.c_int32),
                ("reserved", C.c_int32 * 2)]


SGAD_BWD_WARP_REDUCE = 0
SGAD_BWD_PAIRS = 1
SGAD_BWD_WARP_LOCAL = 2


SGAD_TUNE_PREP = 0
SGAD_TUNE_FWD = 1
SGAD_TUNE_BWD = 2


class sgad_tune_entry(C.Structure):
    _fields_ = [("tile_w", C.c_int32), ("tile_h", C.c_int32), ("stage", C.c_int32), ("batch", C.c_int32),
                ("schedule", C.c_int32), ("ms", C.c_float)]


class sgad_state_view(C.Structure):
    _fields_ = [("tile_offsets", C.c_void_p), ("entries", C.c_void_p), ("t_final", C.c_void_p),
                ("n_contrib", C.c_void_p), ("n_tiles", C.c_int32), ("n_pixels", C.c_int64)]


class sgad_adam_tensor(C.Structure):
    _fields_ = [("param", C.c_void_p), ("grad", C.c_void_p), ("m", C.c_void_p), ("v", C.c_void_p),
                ("n", C.c_int64), ("lr", C.c_float), ("mode", C.c_int32)]


class sgad_stats(C.Structure):
    _fields_ = [("n_keys", C.c_int64), ("keys_needed", C.c_int64), ("n_pairs", C.c_int64),
                ("n_evals", C.c_int64), ("n_sort_exact", C.c_int64)]


SGAD_NET_LAYERS = 4


class sgad_net_params(C.Structure):
    _fields_ = [("w", C.c_void_p * SGAD_NET_LAYERS), ("b", C.c_void_p * SGAD_NET_LAYERS)]


class sgad_net_grads(C.Structure):
    _fields_ = [("dw", C.c_void_p * SGAD_NET_LAYERS), ("db", C.c_void_p * SGAD_NET_LAYERS)]


class sgad_net_buffers(C.Structure):
    _fields_ = [("x", C.c_void_p * 4), ("y4", C.c_void_p), ("dy4", C.c_void_p), ("dpre", C.c_void_p * 3)]


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_needed: bool = True) -> C.CDLL:
    """Load libsgad.so (compiling it first when needed). Raises on any failure."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_needed:
        _build.build()
    if not os.path.exists(_build.LIB):
        raise ImportError("libsgad.so is missing; run paper_2603_21055_gb300.build.build()")
    l = C.CDLL(_build.LIB)
    P, I32, I64 = C.c_void_p, C.c_int32, C.c_int64
    st = C.c_int32
    sig = {
        "sgad_default_options": (st, [P]),
        "sgad_create": (st, [P, P]),
        "sgad_destroy": (None, [P]),
        "sgad_last_error": (C.c_char_p, []),
        "sgad_workspace_size": (st, [P, P, I32, P, I32, I64, P]),
        "sgad_count_keys": (st, [P, P, I32, P, I32, P, C.c_size_t, P, P]),
        "sgad_forward": (st, [P, P, I32, P, I32, P, P, C.c_size_t, I64, P]),
        "sgad_backward": (st, [P, P, I32, P, I32, P, P, P, C.c_size_t, I64, P]),
        "sgad_check": (st, [P, P, C.c_size_t, P, P, P]),
        "sgad_state": (st, [P, P, I32, P, I32, P, C.c_size_t, I64, P]),
        "sgad_read_stats": (st, [P, P, C.c_size_t, P, P]),
        "sgad_profile_enable": (st, [P, I32]),
        "sgad_profile_read": (st, [P, P]),
        "sgad_l1_loss_grad": (st, [I32, P, P, P, P, C.c_float, C.c_float, C.c_float, P, P, P, P, P]),
        "sgad_pose_adam_step": (st, [P, P, P, C.c_float, C.c_float, C.c_float, C.c_float, C.c_float, P]),
        "sgad_adam_step": (st, [I64, P, P, P, P, C.c_float, C.c_float, C.c_float, C.c_float, I32, I32, P]),
        "sgad_adam_step_multi": (st, [I32, P, C.c_float, C.c_float, C.c_float, P, P]),
        "sgad_forward_noalloc": (st, [P, P, I32, P, I32, P, P]),
        "sgad_autotune": (st, [P, P, I32, P, I32, P, P, P, P, C.c_size_t, I32, P, I32, P, P]),
        "sgad_get_options": (st, [P, P]),
        "sgad_ssim_workspace_size": (st, [I32, P, P]),
        "sgad_ssim_loss_grad": (st, [I32, P, P, P, C.c_float, P, P, P, C.c_size_t, P]),
        "sgad_fma_burn": (st, [I32, I32, P, P, P]),
        "sgad_gicp_default_params": (st, [P]),
        "sgad_gicp_workspace_size": (st, [P, P]),
        "sgad_gicp_frame": (st, [P, P, P, P, P, P, P, C.c_size_t, P]),
        "sgad_gicp_index": (st, [P, P, P, C.c_size_t, P]),
        "sgad_gicp_correspond": (st, [P, P, P, P, P, P, C.c_size_t, P]),
        "sgad_gicp_linearize": (st, [P, P, P, P, P, P, C.c_size_t, P]),
        "sgad_gicp_set_pose": (st, [P, P, C.c_size_t, P]),
        "sgad_gicp_track": (st, [P, P, P, P, P, C.c_size_t, P]),
        "sgad_gicp_insert": (st, [P, P, P, P, C.c_size_t, P]),
        "sgad_gicp_result": (st, [P, C.c_size_t, P, P, P]),
        "sgad_net_layer_shape": (st, [I32, P, P, P, P]),
        "sgad_net_workspace_size": (st, [I32, I32, I32, P]),
        "sgad_net_forward": (st, [P, I32, I32, I32, P, P, P, P, P, C.c_size_t, P]),
        "sgad_net_loss_grad": (st, [I32, I32, I32, P, P, C.c_float, P, P, C.c_size_t, P]),
        "sgad_net_backward": (st, [P, P, I32, I32, I32, P, C.c_size_t, P]),
        "sgad_net_check": (st, [P, C.c_size_t, P]),
        "sgad_net_buffers_view": (st, [I32, I32, I32, P, C.c_size_t, P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(l, name)
        f.restype = res
        f.argtypes = args
    _lib = l
    return l


def last_error() -> str:
    return load().sgad_last_error().decode()


def check(status: int) -> None:
    if status != SGAD_OK:
        raise SgadError(status, last_error())


def _call(name, *args):
    check(getattr(load(), name)(*args))


# Same names as the C ABI; arguments are ctypes objects / integers (device addresses).

def sgad_default_options() -> sgad_options:
    o = sgad_options()
    _call("sgad_default_options", C.byref(o))
    return o


def sgad_create(opt: sgad_options | None = None) -> C.c_void_p:
    ctx = C.c_void_p()
    _call("sgad_create", C.byref(ctx), C.byref(opt) if opt is not None else None)
    return ctx


def sgad_destroy(ctx) -> None:
    load().sgad_destroy(ctx)


def sgad_workspace_size(ctx, kfs, views, key_capacity: int) -> int:
    n = C.c_size_t()
    _call("sgad_workspace_size", ctx, kfs, len(kfs), views, len(views), int(key_capacity), C.byref(n))
    return n.value


def sgad_count_keys(ctx, kfs, views, workspace: int, ws_bytes: int, stream: int) -> int:
    n = C.c_int64()
    _call("sgad_count_keys", ctx, kfs, len(kfs), views, len(views), workspace, ws_bytes, C.byref(n), stream)
    return n.value


def sgad_forward(ctx, kfs, views, out, workspace: int, ws_bytes: int, key_capacity: int, stream: int) -> None:
    _call("sgad_forward", ctx, kfs, len(kfs), views, len(views), out, workspace, ws_bytes, int(key_capacity), stream)


def sgad_backward(ctx, kfs, views, grad_in, grads_out, workspace: int, ws_bytes: int, key_capacity: int,
                  stream: int) -> None:
    _call("sgad_backward", ctx, kfs, len(kfs), views, len(views), grad_in, grads_out, workspace, ws_bytes,
          int(key_capacity), stream)


def sgad_check(ctx, workspace: int, ws_bytes: int, stream: int):
    """Returns (status, n_keys, keys_needed) without raising."""
    n, need = C.c_int64(), C.c_int64()
    s = load().sgad_check(ctx, workspace, ws_bytes, C.byref(n), C.byref(need), stream)
    return s, n.value, need.value


def sgad_state(ctx, kfs, views, workspace: int, ws_bytes: int, key_capacity: int) -> sgad_state_view:
    out = sgad_state_view()
    _call("sgad_state", ctx, kfs, len(kfs), views, len(views), workspace, ws_bytes, int(key_capacity),
          C.byref(out))
    return out


def sgad_read_stats(ctx, workspace: int, ws_bytes: int, stream: int) -> sgad_stats:
    out = sgad_stats()
    _call("sgad_read_stats", ctx, workspace, ws_bytes, C.byref(out), stream)
    return out


def sgad_profile_enable(ctx, enable: bool) -> None:
    _call("sgad_profile_enable", ctx, int(bool(enable)))


def sgad_profile_read(ctx):
    ms = (C.c_float * SGAD_NUM_STAGES)()
    _call("sgad_profile_read", ctx, ms)
    return list(ms)


def sgad_l1_loss_grad(views, rendered, target_rgb, target_depth, rgb_weight, depth_weight, d_rgb, d_depth,
                      loss_accum: int, valid_count: int, stream: int, min_alpha: float = -1.0) -> None:
    _call("sgad_l1_loss_grad", len(views), views, rendered, target_rgb, target_depth, float(rgb_weight),
          float(depth_weight), float(min_alpha), d_rgb, d_depth, loss_accum, valid_count, stream)


SGAD_POSE_STATE_FLOATS = 64


def sgad_pose_adam_step(d_pose: int, view_pose, state: int, lr_rot: float, lr_trans: float, beta1: float = 0.9,
                        beta2: float = 0.999, eps: float = 1e-12, stream: int = 0) -> None:
    """view_pose: 12 host floats (row-major 3x4 world->cam); d_pose, state: device pointers."""
    w0 = (C.c_float * 12)(*[float(x) for x in view_pose])
    _call("sgad_pose_adam_step", d_pose, w0, state, float(lr_rot), float(lr_trans), float(beta1), float(beta2),
          float(eps), stream)


def sgad_ssim_workspace_size(views) -> int:
    n = C.c_size_t(0)
    _call("sgad_ssim_workspace_size", len(views), views, C.byref(n))
    return n.value


def sgad_ssim_loss_grad(views, rendered, target_rgb, weight, d_rgb, loss_accum: int, workspace: int,
                        ws_bytes: int, stream: int) -> None:
    _call("sgad_ssim_loss_grad", len(views), views, rendered, target_rgb, float(weight), d_rgb, loss_accum,
          workspace, C.c_size_t(ws_bytes), stream)


def sgad_fma_burn(blocks: int, iters: int, sink: int, stream: int) -> float:
    flops = C.c_double(0.0)
    _call("sgad_fma_burn", int(blocks), int(iters), sink, C.byref(flops), stream)
    return flops.value


def sgad_gicp_default_params() -> sgad_gicp_params:
    p = sgad_gicp_params()
    _call("sgad_gicp_default_params", C.byref(p))
    return p


def sgad_gicp_workspace_size(p: sgad_gicp_params) -> int:
    n = C.c_size_t(0)
    _call("sgad_gicp_workspace_size", C.byref(p), C.byref(n))
    return n.value


def sgad_gicp_frame(p, cam, depth: int, out: sgad_gaussian_set, pix_out: int, knn_out: int, ws: int, ws_bytes: int,
                    stream: int) -> None:
    _call("sgad_gicp_frame", C.byref(p), C.byref(cam), depth, C.byref(out), pix_out or None, knn_out or None, ws,
          C.c_size_t(ws_bytes), stream)


def sgad_gicp_index(p, map_: sgad_gaussian_set, ws: int, ws_bytes: int, stream: int) -> None:
    _call("sgad_gicp_index", C.byref(p), C.byref(map_), ws, C.c_size_t(ws_bytes), stream)


def _f12(pose):
    a = (C.c_float * 12)()
    for i, v in enumerate(list(pose)):
        a[i] = float(v)
    return a


def _d12(pose):
    a = (C.c_double * 12)()
    for i, v in enumerate(list(pose)):
        a[i] = float(v)
    return a


def sgad_gicp_correspond(p, src, map_, pose, idx_out: int, ws: int, ws_bytes: int, stream: int) -> None:
    _call("sgad_gicp_correspond", C.byref(p), C.byref(src), C.byref(map_), _f12(pose), idx_out, ws,
          C.c_size_t(ws_bytes), stream)


def sgad_gicp_linearize(p, src, map_, pose, system_out: int, ws: int, ws_bytes: int, stream: int) -> None:
    _call("sgad_gicp_linearize", C.byref(p), C.byref(src), C.byref(map_), _f12(pose), system_out, ws,
          C.c_size_t(ws_bytes), stream)


def sgad_gicp_set_pose(pose, ws: int, ws_bytes: int, stream: int) -> None:
    _call("sgad_gicp_set_pose", _d12(pose), ws, C.c_size_t(ws_bytes), stream)


def sgad_gicp_track(p, src, map_, pose0, ws: int, ws_bytes: int, stream: int) -> None:
    """pose0 None: start from the workspace's pose."""
    _call("sgad_gicp_track", C.byref(p), C.byref(src), C.byref(map_), _d12(pose0) if pose0 is not None else None, ws,
          C.c_size_t(ws_bytes), stream)


def sgad_gicp_insert(p, src, map_, ws: int, ws_bytes: int, stream: int) -> None:
    _call("sgad_gicp_insert", C.byref(p), C.byref(src), C.byref(map_), ws, C.c_size_t(ws_bytes), stream)


def sgad_gicp_result(ws: int, ws_bytes: int, stream: int):
    pose = (C.c_double * 12)()
    st = sgad_gicp_stats()
    _call("sgad_gicp_result", ws, C.c_size_t(ws_bytes), pose, C.byref(st), stream)
    return list(pose), st


SGAD_ADAM_PLAIN = 0
SGAD_ADAM_LOG = 1


def sgad_adam_step(n: int, param: int, grad: int, m: int, v: int, lr: float, beta1: float, beta2: float,
                   eps: float, step: int, mode: int, stream: int) -> None:
    _call("sgad_adam_step", int(n), param, grad, m, v, float(lr), float(beta1), float(beta2), float(eps),
          int(step), int(mode), stream)


def ptr_array(ptrs):
    """A C array of device pointers (void *) from a list of integers (0 -> NULL)."""
    arr = (C.c_void_p * max(1, len(ptrs)))()
    for i, p in enumerate(ptrs):
        arr[i] = p or None
    return arr


def sgad_adam_step_multi(tensors, beta1: float, beta2: float, eps: float, step_counter: int, stream: int) -> None:
    """tensors: a ctypes array of sgad_adam_tensor; step_counter: device int32 address."""
    _call("sgad_adam_step_multi", len(tensors), tensors, float(beta1), float(beta2), float(eps), step_counter,
          stream)


def sgad_forward_noalloc(ctx, kfs, views, out, stream: int) -> None:
    """Forward splatting into `out` with the library's static scratch (no workspace, no
    allocation); synchronises `stream`."""
    _call("sgad_forward_noalloc", ctx, kfs, len(kfs), views, len(views), out, stream)


def sgad_get_options(ctx) -> sgad_options:
    o = sgad_options()
    _call("sgad_get_options", ctx, C.byref(o))
    return o


def sgad_autotune(ctx, kfs, views, out, grad_in, grads_out, workspace: int, ws_bytes: int, reps: int,
                  stream: int, max_entries: int = 256):
    """Runs the library's autotuner (synchronous); returns its timing rows as dicts."""
    rows = (sgad_tune_entry * max_entries)()
    n = C.c_int32()
    _call("sgad_autotune", ctx, kfs, len(kfs), views, len(views), out, grad_in, grads_out, workspace, ws_bytes,
          int(reps), rows, max_entries, C.byref(n), stream)
    return [dict(tile=(r.tile_w, r.tile_h), stage=("prep", "fwd", "bwd")[r.stage], batch=r.batch,
                 schedule=SCHEDULE_NAMES.get(r.schedule, r.schedule), ms=r.ms) for r in rows[:n.value]]


# ------------------------------------------------------------------ proposal net

def sgad_net_layer_shape(layer: int):
    """(cin, cout, cin_padded, cout_padded) of layer 0..3."""
    v = [C.c_int32() for _ in range(4)]
    _call("sgad_net_layer_shape", int(layer), *[C.byref(x) for x in v])
    return tuple(x.value for x in v)


def sgad_net_workspace_size(n: int, h: int, w: int) -> int:
    b = C.c_size_t()
    _call("sgad_net_workspace_size", int(n), int(h), int(w), C.byref(b))
    return b.value


def sgad_net_forward(params, n, h, w, rgb, depth, delta, logit, workspace, ws_bytes, stream) -> None:
    _call("sgad_net_forward", C.byref(params), int(n), int(h), int(w), rgb, depth, delta or None, logit or None,
          workspace, ws_bytes, stream)


def sgad_net_loss_grad(n, h, w, target_delta, target_logit, logit_weight, loss_accum, workspace, ws_bytes,
                       stream) -> None:
    _call("sgad_net_loss_grad", int(n), int(h), int(w), target_delta, target_logit, float(logit_weight),
          loss_accum or None, workspace, ws_bytes, stream)


def sgad_net_backward(params, grads, n, h, w, workspace, ws_bytes, stream) -> None:
    _call("sgad_net_backward", C.byref(params), C.byref(grads), int(n), int(h), int(w), workspace, ws_bytes,
          stream)


def sgad_net_check(workspace, ws_bytes, stream) -> int:
    """Device status of the net workspace (0 = ok); synchronises; does not raise."""
    return load().sgad_net_check(workspace, ws_bytes, stream)


def sgad_net_buffers_view(n, h, w, workspace, ws_bytes) -> sgad_net_buffers:
    out = sgad_net_buffers()
    _call("sgad_net_buffers_view", int(n), int(h), int(w), workspace, ws_bytes, C.byref(out))
    return out
