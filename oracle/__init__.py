"""FP64 CPU oracle for the splatting of pixel-aligned Gaussians (ctypes front end).

TEST INFRASTRUCTURE ONLY. The oracle is the plain definition of what the CUDA library
computes; only the tests, the package smoke check and the CPU-baseline / reference leg
of the benchmark may load it. It shares no code with the CUDA library and never imports
the package: inputs arrive as duck-typed scene objects (``.keyframes``, ``.views``) holding
the float32 arrays the CUDA path is given; they are upcast exactly to FP64 here (or passed
as float64 by finite-difference tests that perturb them).

The C source (sgad_oracle.c) is compiled with gcc on first use.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sgad_oracle.c")
_HDR = os.path.join(_HERE, "sgad_oracle.h")
_LIB = os.path.join(_HERE, "libsgad_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, -O2, OpenMP) if it is missing or stale."""
    stale = (not os.path.exists(_LIB) or
             os.path.getmtime(_LIB) < max(os.path.getmtime(_SRC), os.path.getmtime(_HDR)))
    if force or stale:
        tmp = _LIB + ".%d.tmp" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp", "-fno-fast-math",
               "-ffp-contract=off", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class Cam(C.Structure):
    _fields_ = [("width", C.c_int32), ("height", C.c_int32), ("fx", C.c_double), ("fy", C.c_double),
                ("cx", C.c_double), ("cy", C.c_double), ("pose", C.c_double * 12)]


class Kf(C.Structure):
    _fields_ = [("cam", Cam), ("depth", C.c_void_p), ("offset", C.c_void_p), ("rgb", C.c_void_p),
                ("logit", C.c_void_p), ("scale", C.c_void_p), ("learnable", C.c_int32)]


class Opts(C.Structure):
    _fields_ = [("tile_w", C.c_int32), ("tile_h", C.c_int32), ("bg", C.c_double * 3),
                ("margin", C.c_double), ("t_margin", C.c_double)]


class Proj(C.Structure):
    _fields_ = [("visible", C.c_int32), ("tx0", C.c_int32), ("tx1", C.c_int32), ("ty0", C.c_int32),
                ("ty1", C.c_int32), ("ntiles", C.c_int32), ("near", C.c_int32), ("pad_", C.c_int32),
                ("mu", C.c_double * 3), ("t", C.c_double * 3), ("p", C.c_double * 2),
                ("cov", C.c_double * 3), ("conic", C.c_double * 3), ("o", C.c_double),
                ("rho", C.c_double), ("zf", C.c_double), ("s", C.c_double), ("color", C.c_double * 3),
                ("pf", C.c_float * 2), ("conicf", C.c_float * 3), ("of", C.c_float)]


class Image(C.Structure):
    _fields_ = [("rgb", C.c_void_p), ("depth", C.c_void_p), ("alpha", C.c_void_p),
                ("t_final", C.c_void_p), ("n_contrib", C.c_void_p), ("near", C.c_void_p)]


class KfGrads(C.Structure):
    _fields_ = [("d_offset", C.c_void_p), ("d_rgb", C.c_void_p), ("d_logit", C.c_void_p),
                ("d_scale", C.c_void_p)]


class ImageGrads(C.Structure):
    _fields_ = [("d_rgb", C.c_void_p), ("d_depth", C.c_void_p), ("d_alpha", C.c_void_p)]


PROJ_DTYPE = np.dtype([("visible", np.int32), ("tx0", np.int32), ("tx1", np.int32), ("ty0", np.int32),
                       ("ty1", np.int32), ("ntiles", np.int32), ("near", np.int32), ("pad_", np.int32),
                       ("mu", np.float64, 3), ("t", np.float64, 3), ("p", np.float64, 2),
                       ("cov", np.float64, 3), ("conic", np.float64, 3), ("o", np.float64),
                       ("rho", np.float64), ("zf", np.float64), ("s", np.float64),
                       ("color", np.float64, 3), ("pf", np.float32, 2), ("conicf", np.float32, 3),
                       ("of", np.float32)])
assert PROJ_DTYPE.itemsize == C.sizeof(Proj)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            l = C.CDLL(build())
            P = C.c_void_p
            l.orc_num_gaussians.restype = C.c_int64
            l.orc_num_gaussians.argtypes = [P, C.c_int32]
            l.orc_num_tiles.restype = C.c_int32
            l.orc_num_tiles.argtypes = [P, C.c_int32, P]
            l.orc_project.argtypes = [P, C.c_int32, P, P, P]
            l.orc_keys.restype = C.c_int64
            l.orc_keys.argtypes = [P, C.c_int32, P, C.c_int32, P, P, P, P]
            l.orc_render.argtypes = [P, C.c_int32, P, C.c_int32, P, P]
            l.orc_render_pixels.argtypes = [P, C.c_int32, P, C.c_int32, P, C.c_int64, P, P, P, P, P, P,
                                            P, P, P]
            l.orc_backward.argtypes = [P, C.c_int32, P, C.c_int32, P, P, P, P, P]
            l.orc_backward_pose.argtypes = [P, C.c_int32, P, C.c_int32, P, P, P, P]
            l.orc_backward_gaussians.argtypes = [P, C.c_int32, P, C.c_int32, P, P, C.c_int64, P, P, P, P]
            l.orc_decision_hash.restype = C.c_uint64
            l.orc_decision_hash.argtypes = [P, C.c_int32, P, C.c_int32, P]
            l.orc_l1_loss.restype = C.c_double
            l.orc_l1_loss.argtypes = [C.c_int32, P, P, P, P, P, C.c_double, C.c_double, P, P]
            l.orc_adam.argtypes = [C.c_int64, P, P, P, P, C.c_double, C.c_double, C.c_double,
                                   C.c_double, C.c_int32, C.c_int32]
            _lib = l
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def _cam(c) -> Cam:
    pose = np.asarray(c.pose, np.float64).reshape(12)
    return Cam(int(c.width), int(c.height), float(c.fx), float(c.fy), float(c.cx), float(c.cy),
               (C.c_double * 12)(*pose))


class _Inputs:
    """FP64 copies of the scene arrays (exact upcasts of float32 inputs, or the caller's
    float64 arrays as they are), kept alive while C holds pointers to them."""

    def __init__(self, scene):
        self.keep = []
        kfs = (Kf * len(scene.keyframes))()
        for i, k in enumerate(scene.keyframes):
            arrs = [np.ascontiguousarray(x, np.float64) for x in (k.depth, k.offset, k.rgb, k.logit, k.scale)]
            self.keep += arrs
            kfs[i] = Kf(_cam(k.cam), *[_ptr(a) for a in arrs], int(bool(k.learnable)))
        views = (Cam * max(1, len(scene.views)))()
        for i, v in enumerate(scene.views):
            views[i] = _cam(v)
        self.kfs, self.n_kf = kfs, len(scene.keyframes)
        self.views, self.n_views = views, len(scene.views)


def opts(tile_w: int = 16, tile_h: int = 16, bg=(0.0, 0.0, 0.0), margin: float = 4e-6,
         t_margin: float = 2e-4) -> Opts:
    """Tile shape, background, and the relative margins under which the single-precision
    alpha decisions (floor, cap) and the transmittance stop are reported near."""
    return Opts(tile_w, tile_h, (C.c_double * 3)(*bg), margin, t_margin)


def num_gaussians(scene) -> int:
    return sum(k.cam.width * k.cam.height for k in scene.keyframes)


def project(scene, view: int, o: Opts = None) -> np.ndarray:
    o = o or opts()
    inp = _Inputs(scene)
    out = np.zeros(num_gaussians(scene), PROJ_DTYPE)
    lib().orc_project(inp.kfs, inp.n_kf, C.byref(inp.views[view]), C.byref(o), _ptr(out))
    return out


def keys(scene, o: Opts = None):
    """Brute-force sorted key list: (keys u64, vals u32, near u8)."""
    o = o or opts()
    inp = _Inputs(scene)
    n = lib().orc_keys(inp.kfs, inp.n_kf, inp.views, inp.n_views, C.byref(o), None, None, None)
    k = np.zeros(n, np.uint64)
    v = np.zeros(n, np.uint32)
    nr = np.zeros(n, np.uint8)
    lib().orc_keys(inp.kfs, inp.n_kf, inp.views, inp.n_views, C.byref(o), _ptr(k), _ptr(v), _ptr(nr))
    return k, v, nr


def render(scene, o: Opts = None):
    """Full forward render of every view: list of dicts of FP64 images."""
    o = o or opts()
    inp = _Inputs(scene)
    outs, imgs = [], (Image * max(1, inp.n_views))()
    for i, v in enumerate(scene.views):
        h, w = v.height, v.width
        d = dict(rgb=np.zeros((3, h, w)), depth=np.zeros((h, w)), alpha=np.zeros((h, w)),
                 t_final=np.zeros((h, w)), n_contrib=np.zeros((h, w), np.int32),
                 near=np.zeros((h, w), np.uint8))
        outs.append(d)
        imgs[i] = Image(*[_ptr(d[k]) for k in ("rgb", "depth", "alpha", "t_final", "n_contrib", "near")])
    lib().orc_render(inp.kfs, inp.n_kf, inp.views, inp.n_views, C.byref(o), imgs)
    return outs


def render_pixels(scene, view_idx, xs, ys, o: Opts = None):
    """Forward render of selected pixels; returns a dict of per-pixel arrays."""
    o = o or opts()
    inp = _Inputs(scene)
    vi = np.ascontiguousarray(view_idx, np.int32)
    x = np.ascontiguousarray(xs, np.int32)
    y = np.ascontiguousarray(ys, np.int32)
    n = vi.shape[0]
    d = dict(rgb=np.zeros((n, 3)), depth=np.zeros(n), alpha=np.zeros(n), t_final=np.zeros(n),
             n_contrib=np.zeros(n, np.int32), near=np.zeros(n, np.uint8))
    lib().orc_render_pixels(inp.kfs, inp.n_kf, inp.views, inp.n_views, C.byref(o), n, _ptr(vi), _ptr(x),
                            _ptr(y), *[_ptr(d[k]) for k in ("rgb", "depth", "alpha", "t_final",
                                                             "n_contrib", "near")])
    return d


def _image_grads(scene, grads_in):
    keep = []
    gi = (ImageGrads * max(1, len(scene.views)))()
    for i, v in enumerate(scene.views):
        h, w = v.height, v.width
        g = grads_in[i]
        arrs = [np.ascontiguousarray(np.broadcast_to(np.asarray(g.get(k, 0.0), np.float64), s))
                for k, s in (("rgb", (3, h, w)), ("depth", (h, w)), ("alpha", (h, w)))]
        keep += arrs
        gi[i] = ImageGrads(*[_ptr(a) for a in arrs])
    return gi, keep


def backward(scene, grads_in, o: Opts = None):
    """Adjoint of the render. grads_in: per view dict with 'rgb' (3,H,W), 'depth',
    'alpha' (missing entries are zero). Returns per keyframe dict d_offset, d_rgb,
    d_logit, d_scale (zeros for fixed keyframes), 'near' (H, W): Gaussians reached by a
    pixel with a near decision, whose gradient FP32 may legitimately change, and 'abs':
    per attribute the sum over views and pixels of |each pixel's contribution|."""
    o = o or opts()
    inp = _Inputs(scene)
    gi, keep = _image_grads(scene, grads_in)
    outs, gk = [], (KfGrads * max(1, inp.n_kf))()
    for i, k in enumerate(scene.keyframes):
        h, w = k.cam.height, k.cam.width
        d = dict(d_offset=np.zeros((h, w)), d_rgb=np.zeros((3, h, w)), d_logit=np.zeros((h, w)),
                 d_scale=np.zeros((h, w)))
        outs.append(d)
        gk[i] = KfGrads(*[_ptr(d[q]) for q in ("d_offset", "d_rgb", "d_logit", "d_scale")])
    near = np.zeros(num_gaussians(scene), np.uint8)
    absum = np.zeros((num_gaussians(scene), 6))
    lib().orc_backward(inp.kfs, inp.n_kf, inp.views, inp.n_views, C.byref(o), gi, gk, _ptr(near), _ptr(absum))
    base = 0
    for d, k in zip(outs, scene.keyframes):
        n = k.cam.width * k.cam.height
        h, w = k.cam.height, k.cam.width
        d["near"] = near[base:base + n].reshape(h, w).astype(bool)
        a = absum[base:base + n]
        d["abs"] = dict(d_offset=a[:, 0].reshape(h, w), d_rgb=a[:, 1:4].T.reshape(3, h, w),
                        d_logit=a[:, 4].reshape(h, w), d_scale=a[:, 5].reshape(h, w))
        base += n
    del keep
    return outs


def backward_pose(scene, grads_in, o: Opts = None):
    """Adjoint into the view poses: (d_pose, abs) as (n_views, 3, 4) arrays, d loss / d of
    each view's world->cam 3x4 matrix and the sum of the magnitudes of the per-pixel
    contributions."""
    o = o or opts()
    inp = _Inputs(scene)
    gi, keep = _image_grads(scene, grads_in)
    nv = len(scene.views)
    d = np.zeros((nv, 12))
    a = np.zeros((nv, 12))
    lib().orc_backward_pose(inp.kfs, inp.n_kf, inp.views, inp.n_views, C.byref(o), gi, _ptr(d), _ptr(a))
    del keep
    return d.reshape(nv, 3, 4), a.reshape(nv, 3, 4)


def backward_gaussians(scene, grads_in, sel, o: Opts = None):
    """Adjoint for selected global Gaussian indices: ((n, 6) array of (d_offset, d_r, d_g,
    d_b, d_logit, d_scale), (n,) bool near flags and (n, 6) contribution magnitudes as in
    backward())."""
    o = o or opts()
    inp = _Inputs(scene)
    gi, keep = _image_grads(scene, grads_in)
    s = np.ascontiguousarray(sel, np.int64)
    out = np.zeros((s.shape[0], 6))
    near = np.zeros(s.shape[0], np.uint8)
    absum = np.zeros((s.shape[0], 6))
    lib().orc_backward_gaussians(inp.kfs, inp.n_kf, inp.views, inp.n_views, C.byref(o), gi, s.shape[0],
                                 _ptr(s), _ptr(out), _ptr(near), _ptr(absum))
    del keep
    return out, near.astype(bool), absum


def decision_hash(scene, o: Opts = None) -> int:
    o = o or opts()
    inp = _Inputs(scene)
    return int(lib().orc_decision_hash(inp.kfs, inp.n_kf, inp.views, inp.n_views, C.byref(o)))


def l1_loss(scene, renders):
    """Eq. 1 L1 terms (no SSIM) against the scene's targets; returns (loss, per-view
    dicts of d loss / d rgb and d loss / d depth)."""
    inp = _Inputs(scene)
    nv = len(scene.views)
    keep, grads = [], []
    P = C.c_void_p
    rgb_p, dep_p, trgb_p, tdep_p, drgb_p, ddep_p = [(P * max(1, nv))() for _ in range(6)]
    for i in range(nv):
        r = np.ascontiguousarray(renders[i]["rgb"], np.float64)
        d = np.ascontiguousarray(renders[i]["depth"], np.float64)
        tr = np.ascontiguousarray(scene.target_rgb[i], np.float64)
        td = np.ascontiguousarray(scene.target_depth[i], np.float64)
        g = dict(rgb=np.zeros_like(r), depth=np.zeros_like(d))
        keep += [r, d, tr, td]
        grads.append(g)
        rgb_p[i], dep_p[i], trgb_p[i], tdep_p[i] = _ptr(r), _ptr(d), _ptr(tr), _ptr(td)
        drgb_p[i], ddep_p[i] = _ptr(g["rgb"]), _ptr(g["depth"])
    loss = lib().orc_l1_loss(nv, inp.views, rgb_p, dep_p, trgb_p, tdep_p, float(scene.rgb_weight),
                             float(scene.depth_weight), drgb_p, ddep_p)
    return loss, grads


def adam(param, grad, m, v, lr, beta1=0.9, beta2=0.999, eps=1e-15, step=1, log_param=False):
    """One FP64 Adam step in place on float64 arrays (log_param: param holds exp(p))."""
    arrs = [param, grad, m, v]
    for a in arrs:
        assert a.dtype == np.float64 and a.flags.c_contiguous
    lib().orc_adam(param.size, _ptr(param), _ptr(grad), _ptr(m), _ptr(v), lr, beta1, beta2, eps, step,
                   int(bool(log_param)))
