"""CPU-side checks of the C ABI: the library builds and loads, exports every function
include/sgad.h declares, and the host-only calls validate their arguments. No call here
touches a GPU."""
import ctypes as C
import os
import re

import pytest

from paper_2603_21055_gb300 import binding as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    inc = os.path.join(ROOT, "include")
    src = "".join(open(os.path.join(inc, f)).read() for f in sorted(os.listdir(inc)) if f.endswith(".h"))
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sgad_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_function():
    lib = B.load()
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(B.EXPORTS) == names


def test_default_options_and_create():
    o = B.sgad_default_options()
    assert (o.tile_w, o.tile_h) == (16, 16) and o.freeze_offset == 0
    assert (o.fwd_batch, o.bwd_batch) == (512, 256)
    assert o.fwd_schedule == o.bwd_schedule == B.SGAD_SCHEDULE_TILES
    assert o.bwd_algorithm == B.SGAD_BWD_WARP_LOCAL
    ctx = B.sgad_create(o)
    B.sgad_destroy(ctx)
    for w, h in ((8, 32), (32, 8)):
        o.tile_w, o.tile_h = w, h
        B.sgad_destroy(B.sgad_create(o))


def test_work_split_options_round_trip():
    """Every batch size and schedule is accepted and read back unchanged; 0 batches take
    the defaults."""
    for fb in B.FWD_BATCH_SIZES:
        for sched in (B.SGAD_SCHEDULE_TILES, B.SGAD_SCHEDULE_PERSISTENT, B.SGAD_SCHEDULE_PER_VIEW):
            o = B.sgad_default_options()
            o.fwd_batch, o.bwd_batch, o.fwd_schedule, o.bwd_schedule = fb, B.BATCH_SIZES[-1], sched, sched
            ctx = B.sgad_create(o)
            r = B.sgad_get_options(ctx)
            assert (r.fwd_batch, r.bwd_batch, r.fwd_schedule, r.bwd_schedule) == (fb, 512, sched, sched)
            B.sgad_destroy(ctx)
    o = B.sgad_default_options()
    o.fwd_batch = o.bwd_batch = 0
    ctx = B.sgad_create(o)
    r = B.sgad_get_options(ctx)
    assert (r.fwd_batch, r.bwd_batch) == (512, 256)
    B.sgad_destroy(ctx)


def test_autotune_validates_on_the_host():
    ctx = B.sgad_create()
    lib = B.load()
    n = C.c_int32(-1)
    assert lib.sgad_autotune(ctx, None, 1, None, 1, None, None, None, None, 0, 0, None, 0, C.byref(n),
                             None) == B.SGAD_ERR_INVALID_ARG
    assert n.value == 0 and "reps" in B.last_error()
    assert lib.sgad_autotune(None, None, 1, None, 1, None, None, None, None, 0, 3, None, 0, None,
                             None) == B.SGAD_ERR_INVALID_ARG
    B.sgad_destroy(ctx)


@pytest.mark.parametrize("field,value,status", [
    ("tile_w", 12, B.SGAD_ERR_UNSUPPORTED),
    ("sort_smem_cap", 8, B.SGAD_ERR_INVALID_ARG),
    ("fwd_batch", 100, B.SGAD_ERR_UNSUPPORTED),
    ("fwd_batch", 2048, B.SGAD_ERR_UNSUPPORTED),
    ("bwd_batch", 1024, B.SGAD_ERR_UNSUPPORTED),
    ("fwd_schedule", 3, B.SGAD_ERR_INVALID_ARG),
    ("bwd_schedule", -1, B.SGAD_ERR_INVALID_ARG),
    ("bwd_algorithm", 3, B.SGAD_ERR_INVALID_ARG),
    ("max_blocks", -1, B.SGAD_ERR_INVALID_ARG),
])
def test_create_rejects_bad_options(field, value, status):
    o = B.sgad_default_options()
    setattr(o, field, value)
    with pytest.raises(B.SgadError) as e:
        B.sgad_create(o)
    assert e.value.status == status
    assert B.last_error()


def _cam(w=64, h=48):
    c = B.sgad_camera(w, h, 60.0, 60.0, 32.0, 24.0)
    for i, v in enumerate([1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0]):
        c.pose[i] = v
    return c


def test_workspace_size_arithmetic():
    """Workspace = header + 64 B per Gaussian + tile offsets/counters/order/sort list + 8 B per view
    pixel + 16 B per key of key arrays + 32 B per key (+ 1 KB per tile) of contribution
    words + one word per 4 keys (+ 16 per tile and 8) of per-warp contribution masks, each
    section rounded to 256 B."""
    ctx = B.sgad_create()
    kfs = (B.sgad_keyframe * 1)()
    kfs[0].cam = _cam()
    views = (B.sgad_camera * 2)(_cam(), _cam(100, 70))
    n0 = B.sgad_workspace_size(ctx, kfs, views, 0)
    n1 = B.sgad_workspace_size(ctx, kfs, views, 1000)
    r = lambda x: (x + 255) // 256 * 256
    tiles = 4 * 3 + 7 * 5
    # two 8-byte key arrays, 32 bytes of contribution words per key, the mask words
    masks = r(4 * ((1000 >> 2) + 16 * (tiles + 1) + 8)) - r(4 * (16 * (tiles + 1) + 8))
    assert n1 - n0 == 2 * r(1000 * 8) + 1000 * 32 + masks
    ng, npx = 64 * 48, 64 * 48 + 100 * 70
    assert n0 >= 256 + 64 * ng + 8 * npx
    B.sgad_destroy(ctx)


def test_host_validation_without_gpu():
    ctx = B.sgad_create()
    lib = B.load()
    kfs = (B.sgad_keyframe * 1)()
    kfs[0].cam = _cam()
    views = (B.sgad_camera * 1)(_cam())
    n = C.c_size_t()
    assert lib.sgad_workspace_size(ctx, kfs, 0, views, 1, 0, C.byref(n)) == B.SGAD_ERR_INVALID_ARG
    assert lib.sgad_workspace_size(ctx, kfs, 1, views, 65, 0, C.byref(n)) == B.SGAD_ERR_INVALID_ARG
    bad = (B.sgad_camera * 1)(_cam())
    bad[0].fx = -1.0
    assert lib.sgad_workspace_size(ctx, kfs, 1, bad, 1, 0, C.byref(n)) == B.SGAD_ERR_INVALID_ARG
    assert lib.sgad_workspace_size(ctx, kfs, 1, views, 1, -5, C.byref(n)) == B.SGAD_ERR_INVALID_ARG
    assert lib.sgad_adam_step(10, None, None, None, None, 0.1, 0.9, 0.999, 1e-15, 1, 0, None) == B.SGAD_ERR_INVALID_ARG
    B.sgad_destroy(ctx)


def test_net_shapes_and_workspace_on_the_host():
    assert [B.sgad_net_layer_shape(l) for l in range(4)] == [(4, 32, 16, 32), (32, 32, 32, 32), (32, 32, 32, 32),
                                                            (32, 2, 32, 16)]
    n1 = B.sgad_net_workspace_size(1, 48, 64)
    n2 = B.sgad_net_workspace_size(2, 48, 64)
    # per pixel: packed input 32 B, three activations 3 x 64 B, outputs 8 B, output gradient
    # 32 B, three pre-activation gradients 3 x 64 B
    assert n2 - n1 == 48 * 64 * (32 + 192 + 8 + 32 + 192)
    lib = B.load()
    n = C.c_size_t()
    assert lib.sgad_net_workspace_size(0, 48, 64, C.byref(n)) == B.SGAD_ERR_INVALID_ARG
    assert lib.sgad_net_layer_shape(4, None, None, None, None) == B.SGAD_ERR_INVALID_ARG
    p = B.sgad_net_params()
    assert lib.sgad_net_forward(C.byref(p), 1, 48, 64, None, None, None, None, None, 0, None) == B.SGAD_ERR_INVALID_ARG


def test_ssim_workspace_and_validation_on_the_host():
    """SSIM scratch: 9 floats per pixel per view, each view's block rounded to 256 B; bad
    arguments are refused before any launch."""
    views = (B.sgad_camera * 2)(_cam(), _cam(100, 70))
    r = lambda x: (x + 255) // 256 * 256
    assert B.sgad_ssim_workspace_size(views) == r(9 * 4 * 64 * 48) + r(9 * 4 * 100 * 70)
    lib = B.load()
    n = C.c_size_t()
    assert lib.sgad_ssim_workspace_size(0, views, C.byref(n)) == B.SGAD_ERR_INVALID_ARG
    assert lib.sgad_ssim_workspace_size(65, views, C.byref(n)) == B.SGAD_ERR_INVALID_ARG
    bad = (B.sgad_camera * 1)(_cam(0, 10))
    assert lib.sgad_ssim_workspace_size(1, bad, C.byref(n)) == B.SGAD_ERR_INVALID_ARG
    one = (B.sgad_camera * 1)(_cam())
    rend = (B.sgad_images * 1)()
    arr = B.ptr_array([0])
    # NULL images, a missing workspace, a misaligned one and a non-finite weight
    assert lib.sgad_ssim_loss_grad(1, one, rend, arr, C.c_float(0.2), arr, None, None, 0, None) == B.SGAD_ERR_INVALID_ARG
    assert lib.sgad_ssim_loss_grad(1, one, None, arr, C.c_float(0.2), arr, None, None, 0, None) == B.SGAD_ERR_INVALID_ARG
    fake = B.ptr_array([4096])
    rend[0] = B.sgad_images(4096, 0, 0)
    need = B.sgad_ssim_workspace_size(one)
    assert lib.sgad_ssim_loss_grad(1, one, rend, fake, C.c_float(0.2), fake, None, None, need,
                                   None) == B.SGAD_ERR_WORKSPACE_TOO_SMALL
    assert lib.sgad_ssim_loss_grad(1, one, rend, fake, C.c_float(0.2), fake, None, 4096 + 16, need,
                                   None) == B.SGAD_ERR_INVALID_ARG
    assert lib.sgad_ssim_loss_grad(1, one, rend, fake, C.c_float(float("inf")), fake, None, 4096, need,
                                   None) == B.SGAD_ERR_INVALID_ARG


def test_gicp_params_workspace_and_validation_on_the_host():
    p = B.sgad_gicp_default_params()
    assert (p.stride, p.k_cov, p.k_match, p.max_iters) == (10, 10, 5, 30)
    assert abs(p.r_max - 0.1) < 1e-7 and abs(p.d_overlap - 0.02) < 1e-7
    assert (p.src_capacity, p.map_capacity) == (1 << 16, 1 << 20)
    sizes = []
    for src, mp in ((1000, 5000), (2000, 5000), (1000, 10000)):
        p.src_capacity, p.map_capacity = src, mp
        sizes.append(B.sgad_gicp_workspace_size(p))
    assert sizes[1] > sizes[0] and sizes[2] > sizes[0]
    lib = B.load()
    n = C.c_size_t()
    for field, bad in (("stride", 0), ("k_cov", 2), ("k_cov", 33), ("k_match", 9), ("max_iters", 0),
                       ("r_max", 0.0), ("eps", 0.0), ("eps", 2.0), ("src_capacity", 0), ("map_capacity", 1 << 25)):
        q = B.sgad_gicp_default_params()
        setattr(q, field, bad)
        assert lib.sgad_gicp_workspace_size(C.byref(q), C.byref(n)) == B.SGAD_ERR_INVALID_ARG, field
    p = B.sgad_gicp_default_params()
    s = B.sgad_gaussian_set(4096, 4096, 4096, 4096, 0)               # capacity 0
    assert lib.sgad_gicp_index(C.byref(p), C.byref(s), None, 0, None) == B.SGAD_ERR_INVALID_ARG
    s.capacity = 10
    assert lib.sgad_gicp_index(C.byref(p), C.byref(s), None, 0, None) == B.SGAD_ERR_INVALID_ARG    # no workspace
    s.pos = 4100                                                     # misaligned
    assert lib.sgad_gicp_index(C.byref(p), C.byref(s), 4096, 1 << 20, None) == B.SGAD_ERR_INVALID_ARG
    s.pos = 4096
    assert lib.sgad_gicp_index(C.byref(p), C.byref(s), 4096, 16, None) == B.SGAD_ERR_WORKSPACE_TOO_SMALL
    s.capacity = p.map_capacity + 1                                  # above the workspace's capacity
    assert lib.sgad_gicp_index(C.byref(p), C.byref(s), 4096, 1 << 30, None) == B.SGAD_ERR_INVALID_ARG
    cam = B.sgad_camera(0, 10, 100.0, 100.0, 0.0, 0.0)
    assert lib.sgad_gicp_frame(C.byref(p), C.byref(cam), 4096, C.byref(s), None, None, 4096, 1 << 20,
                               None) == B.SGAD_ERR_INVALID_ARG
    nanpose = (C.c_double * 12)(*([float("nan")] * 12))
    assert lib.sgad_gicp_set_pose(nanpose, 4096, 1 << 20, None) == B.SGAD_ERR_INVALID_ARG


def test_fma_probe_validation_on_the_host():
    lib = B.load()
    d = C.c_double()
    assert lib.sgad_fma_burn(0, 10, 4096, C.byref(d), None) == B.SGAD_ERR_INVALID_ARG
    assert lib.sgad_fma_burn(10, 0, 4096, C.byref(d), None) == B.SGAD_ERR_INVALID_ARG
    assert lib.sgad_fma_burn(10, 10, None, C.byref(d), None) == B.SGAD_ERR_INVALID_ARG
