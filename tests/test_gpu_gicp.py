"""GPU parity of the geometric tracking (sgad_gicp_*) against the oracle (oracle/gicp.py).

Integer decisions are compared bit for bit on identical inputs: the selected pixels and
their back-projected points, each point's K_c neighbours, the correspondences at a given
pose and the Gaussians the map update keeps. Floating-point results are compared within
bounds derived from FP32 arithmetic: normalised covariances (entries <= 1) within 2e-3
absolute — the FP32 covariance of ~10 points carries ~1e-6 relative error, amplified by
up to 1 / (eigen-gap) in the eigenvectors (cases with a gap below 1.5x, or nearly
collinear neighbours, are excluded for the normal, whose direction is then not
determined); the Gauss-Newton system within
1e-3 of its largest entry (FP32 per-correspondence terms and block sums against FP64);
tracked poses within 1e-4 m and 0.005 degree of the oracle's from the same inputs.
"""
import math

import numpy as np
import pytest

from oracle import gicp as G

pytestmark = pytest.mark.gpu

W, H, F, CX, CY = 160, 120, 150.0, 80.0, 60.0


def _motion(k):
    """The k-th frame's motion from frame 0: k x (0.8 degree about a fixed axis, 1.5 cm)."""
    from paper_2603_21055_gb300 import synth
    axis = np.array([0.3, 1.0, 0.2])
    return synth.rotation_about(axis / np.linalg.norm(axis), math.radians(0.8 * k)), np.array([0.012, -0.004, 0.008]) * k


@pytest.fixture(scope="module")
def seq():
    """Depth frames of a ray-cast room along a constant-velocity path, with sensor noise
    (1 mm), 2 mm quantisation and a patch of missing depth."""
    from paper_2603_21055_gb300 import synth
    rng = np.random.default_rng(41)
    centre = np.array([3.0, 2.5, 1.5])
    room = synth.make_room(rng, keep_free=(centre, 1.1))
    c2w0 = synth.keyframe_path(rng, 1, centre)[0]
    poses, depths = [], []
    for k in range(6):
        Rm, tm = _motion(k)
        P = np.hstack([Rm @ c2w0[:, :3], (Rm @ c2w0[:, 3] + tm)[:, None]])
        d, _ = synth.raycast(room, P, W, H, F, F, CX, CY)
        d = d + rng.normal(scale=0.001, size=d.shape)
        d = (np.round(d / 0.002) * 0.002).astype(np.float32)
        d[20:35, 100:130] = 0.0
        poses.append(P)
        depths.append(d)
    return poses, depths


def _cam():
    from paper_2603_21055_gb300.synth import Camera
    return Camera(W, H, F, F, CX, CY, np.eye(4, dtype=np.float32)[:3].copy())


def _tracker(**kw):
    from paper_2603_21055_gb300.gicp import GicpTracker
    return GicpTracker(src_capacity=kw.pop("src_capacity", 8192), map_capacity=kw.pop("map_capacity", 65536), **kw)


@pytest.mark.parametrize("stride,k_cov", [(2, 10), (3, 23), (4, 32), (2, 3)])
def test_frame_gaussians_match_oracle(seq, stride, k_cov):
    import torch
    _, depths = seq
    tr = _tracker(stride=stride, k_cov=k_cov)
    knn = torch.full((tr.src.capacity, k_cov), -1, dtype=torch.int32, device="cuda")
    tr.frame(_cam(), torch.as_tensor(depths[0]).cuda(), knn_out=knn)
    torch.cuda.synchronize()
    ref = G.frame_gaussians(depths[0], F, F, CX, CY, stride, k_cov)
    n = tr.src.n()
    assert n == len(ref["points"]) > 0
    pos, cov, nrm = tr.src.host()
    assert np.array_equal(pos, ref["points"])                          # bit-exact back-projection
    assert np.array_equal(tr.pix[:n].cpu().numpy(), ref["pix"])
    assert np.array_equal(knn[:n].cpu().numpy(), ref["knn"])            # neighbours, nearest first
    assert np.abs(cov - ref["cov"]).max() < 2e-3
    s = ref["scales"]
    # the normal is determined where the smallest scale is separated from the middle one
    # and the points are not (nearly) collinear
    gap = (s[:, 1] > 1.5 * s[:, 0]) & (s[:, 1] > 1e-2 * s[:, 2])
    assert gap.mean() > 0.5
    dots = np.abs(np.sum(nrm * ref["normal"], 1))
    assert dots[gap].min() > 0.999


def _oracle_map(depth, pose, stride=2, k_cov=10, d_ov=0.02):
    fg = G.frame_gaussians(depth, F, F, CX, CY, stride, k_cov)
    return G.insert(G.empty_map(), fg, pose, d_ov)


def test_correspondences_and_system_match_oracle(seq):
    import torch
    poses, depths = seq
    tr = _tracker(stride=2, k_cov=10)
    mp = _oracle_map(depths[0], poses[0])
    tr.map.load(mp["points"], mp["cov"], mp["normal"])
    tr.index()
    tr.frame(_cam(), torch.as_tensor(depths[1]).cuda())
    torch.cuda.synchronize()
    spos, scov, _ = tr.src.host()
    map_pos, map_cov, map_nrm = tr.map.host()                         # the exact arrays the GPU sees
    for k, pose in enumerate([poses[1], poses[0], np.hstack([poses[1][:, :3], poses[1][:, 3:] + 0.01])]):
        P32 = np.asarray(pose, np.float32)
        idx = torch.full((tr.src.capacity,), -7, dtype=torch.int32, device="cuda")
        tr.correspond(P32, idx)
        got = idx[:len(spos)].cpu().numpy()
        want = G.correspond(spos, P32, map_pos, map_nrm, 0.1, 5)
        assert (want >= 0).sum() > 0.5 * len(spos), k
        assert np.array_equal(got, want), (k, np.nonzero(got != want)[0][:10])
        sysv = tr.linearize(P32)
        Hr, gr, cost, n = G.gn_system(spos, scov, map_pos, map_cov, want, P32.astype(np.float64))
        Hg = np.zeros((6, 6))
        t = 0
        for r in range(6):
            for c in range(r, 6):
                Hg[r, c] = Hg[c, r] = sysv[t]
                t += 1
        assert int(sysv[28]) == n
        assert np.abs(Hg - Hr).max() <= 1e-3 * np.abs(Hr).max(), k
        assert np.abs(sysv[21:27] - gr).max() <= 1e-3 * max(np.abs(gr).max(), 1e-3 * np.abs(Hr).max()), k
        assert abs(sysv[27] - cost) <= 1e-3 * max(cost, 1e-6), k


def _rot_err_deg(A, B):
    return float(np.degrees(np.arccos(np.clip((np.trace(A[:, :3] @ B[:, :3].T) - 1) / 2, -1, 1))))


def test_tracking_matches_oracle_and_truth(seq):
    import torch
    poses, depths = seq
    tr = _tracker(stride=2, k_cov=10, max_iters=40, tol=1e-7)
    mp = _oracle_map(depths[0], poses[0])
    tr.map.load(mp["points"], mp["cov"], mp["normal"])
    tr.index()
    tr.frame(_cam(), torch.as_tensor(depths[1]).cuda())
    tr.track(poses[0])                                                  # zero-motion start, 1.5 cm / 0.8 deg away
    got, st = tr.result()
    assert st.status & 2 == 0 and st.iterations >= 2
    spos, scov, snrm = tr.src.host()
    map_pos, map_cov, map_nrm = tr.map.host()
    ref = G.gicp(dict(points=spos, cov=scov), dict(points=map_pos, cov=map_cov, normal=map_nrm), poses[0],
                 r_max=0.1, max_iters=40, tol=1e-7)
    assert np.linalg.norm(got[:, 3] - ref[:, 3]) < 1e-4 and _rot_err_deg(got, ref) < 5e-3
    assert np.linalg.norm(got[:, 3] - poses[1][:, 3]) < 5e-3 and _rot_err_deg(got, poses[1]) < 0.1


def test_map_update_matches_oracle(seq):
    import torch
    poses, depths = seq
    tr = _tracker(stride=2, k_cov=10)
    mp = _oracle_map(depths[0], poses[0])
    tr.map.load(mp["points"], mp["cov"], mp["normal"])
    tr.index()
    n0 = tr.map.n()
    tr.frame(_cam(), torch.as_tensor(depths[2]).cuda())
    tr.set_pose(poses[2])
    tr.insert()
    torch.cuda.synchronize()
    spos, scov, snrm = tr.src.host()
    map_pos, _, _ = tr.map.host()
    ref = G.insert(dict(points=map_pos[:n0], cov=np.zeros((n0, 3, 3)), normal=np.zeros((n0, 3))),
                   dict(points=spos, cov=scov, normal=snrm), poses[2], 0.02)
    assert tr.map.n() == n0 + len(ref["added"]) and 0 < len(ref["added"]) < len(spos)
    assert np.array_equal(map_pos, ref["points"])                       # same Gaussians, same order, bit-exact
    _, cov, nrm = tr.map.host()
    np.testing.assert_allclose(cov[n0:], ref["cov"][n0:], atol=1e-5)
    np.testing.assert_allclose(nrm[n0:], ref["normal"][n0:], atol=1e-5)


def test_sequence_tracking(seq):
    import torch
    poses, depths = seq
    tr = _tracker(stride=2, k_cov=10)
    est = tr.track_sequence(_cam(), [torch.as_tensor(d).cuda() for d in depths], poses[0])
    for k in range(1, len(poses)):
        assert np.linalg.norm(est[k][:, 3] - poses[k][:, 3]) < 5e-3, k
        assert _rot_err_deg(est[k], poses[k]) < 0.15, k
    _, st = tr.result()
    assert st.status == 0 and tr.map.n() > tr.src.n()


def test_degenerate_inputs_end_cleanly(seq):
    import torch
    poses, depths = seq
    tr = _tracker(stride=2, k_cov=10, src_capacity=100)
    tr.frame(_cam(), torch.as_tensor(depths[0]).cuda())               # more pixels than the capacity
    tr.set_pose(poses[0])
    _, st = tr.result()
    assert tr.src.n() == 100 and st.status & 1
    tr2 = _tracker(stride=2, k_cov=10)
    tr2.frame(_cam(), torch.zeros(H, W, device="cuda"))                 # no valid depth
    assert tr2.src.n() == 0
    tr2.index()
    tr2.track(poses[0])                                                 # nothing to match: ends at once
    pose, st2 = tr2.result()
    assert st2.status & 2 and st2.iterations == 0
    assert np.allclose(pose, poses[0])


def test_graph_replay_matches_eager_calls(seq):
    """A frame's calls captured once as a CUDA graph and replayed per frame (with the
    starting pose set in the workspace) give the eager calls' poses."""
    import torch
    poses, depths = seq
    eager = _tracker(stride=2, k_cov=10)
    est_e = eager.track_sequence(_cam(), [torch.as_tensor(d).cuda() for d in depths], poses[0])
    tr = _tracker(stride=2, k_cov=10)
    tr.capture(_cam(), H, W)
    tr.frame(_cam(), torch.as_tensor(depths[0]).cuda())
    tr.set_pose(poses[0])
    tr.insert()
    est = [np.asarray(poses[0], np.float64)]
    for i in range(1, len(depths)):
        from paper_2603_21055_gb300.gicp import pose44
        guess = (pose44(est[-1]) @ np.linalg.inv(pose44(est[-2])) @ pose44(est[-1]))[:3] if i >= 2 else est[-1]
        tr.step(torch.as_tensor(depths[i]).cuda(), guess)
        pose, _ = tr.result()
        est.append(pose)
    for a, b in zip(est, est_e):
        assert np.abs(a - b).max() < 1e-9
    assert tr.map.n() == eager.map.n()
