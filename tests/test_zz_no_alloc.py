"""The no-allocation forward entry point (sgad_forward_noalloc) for callers that cannot
allocate device memory: called twice in a row through the C ABI on two different
problems, each time it must give, bit for bit, the images the workspace-based sgad_forward
gives (the same kernels, options and inputs: any difference would come from stale or
short scratch), and
a problem too large for its static scratch must be refused before anything runs.

Kept in a file of its own that pytest collects last."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _render_both(scene):
    import torch
    from paper_2603_21055_gb300 import binding as B
    from paper_2603_21055_gb300 import splat
    sp = splat.Splatter()
    kfs = splat.upload_keyframes(scene)
    sp.plan(kfs, scene.views)
    ref = splat.alloc_images(scene.views)
    sp.forward(kfs, scene.views, ref)
    got = splat.alloc_images(scene.views)
    for im in got:
        for t in im.values():
            t.fill_(float("nan"))
    out = (B.sgad_images * len(scene.views))()
    for i, im in enumerate(got):
        out[i] = B.sgad_images(im["rgb"].data_ptr(), im["depth"].data_ptr(), im["alpha"].data_ptr())
    B.sgad_forward_noalloc(sp.ctx, sp.kf_structs(kfs), sp.view_structs(scene.views), out, sp.stream())
    torch.cuda.synchronize()
    return ref, got


def test_noalloc_forward_matches_workspace_forward_twice(scene1, room2):
    from paper_2603_21055_gb300.synth import crop_scene
    # first call: the 64x48 plane; second call: a different, larger problem, so stale
    # contents of the shared static scratch from the first call would show up
    crop = crop_scene(room2, (200, 150, 160, 120), (190, 140, 176, 130), n_keyframes=2, n_views=2)
    for scene in (scene1, crop):
        ref, got = _render_both(scene)
        for r, g in zip(ref, got):
            for q in ("rgb", "depth", "alpha"):
                a, b = g[q].cpu().numpy(), r[q].cpu().numpy()
                assert np.all(np.isfinite(a)), q
                np.testing.assert_array_equal(a, b, err_msg=q)


def test_noalloc_refuses_problems_beyond_its_scratch(room2):
    from paper_2603_21055_gb300 import binding as B
    from paper_2603_21055_gb300 import splat
    sp = splat.Splatter()
    kfs = splat.upload_keyframes(room2)                # 2.46M Gaussians: > 64 MiB of scratch
    out = (B.sgad_images * len(room2.views))()
    st = B.load().sgad_forward_noalloc(sp.ctx, sp.kf_structs(kfs), len(kfs), sp.view_structs(room2.views),
                                       len(room2.views), out, None)
    assert st == B.SGAD_ERR_WORKSPACE_TOO_SMALL
    assert "static scratch" in B.last_error()
