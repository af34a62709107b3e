"""The frame-sharded mapping schedule on CPU ranks (gloo, world size 2): waves, the
all-gather of each wave's parameters, which neighbours a frame sees as fixed, a last wave
shorter than the world, and the own-only mode. The per-frame mapping is replaced by a
stand-in whose result depends on the frame and on every fixed neighbour it was given, so
a wrong exchange or schedule changes the numbers."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2603_21055_gb300 import parallel as P

HW = 6                      # a 3 x 2 "image": 36 floats per frame


def stand_in(i, fixed):
    """Frame i's 'mapped' parameters: a frame-specific pattern plus 0.5 x each fixed
    neighbour (only neighbours of i count)."""
    out = torch.arange(P.N_PLANES * HW, dtype=torch.float32) * 1e-3 + float(i)
    for j in P.neighbours(i):
        if j in fixed:
            out = out + 0.5 * fixed[j]
    return out


def schedule_by_hand(n_frames, world, own_only):
    """The same schedule computed in one process: a frame sees the frames of earlier
    waves only."""
    params = {}
    for wave in P.waves(n_frames, world):
        fixed = {} if own_only else dict(params)
        outs = {i: stand_in(i, fixed) for i in wave}
        params.update(outs)
    return params


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, n_frames, own_only, out_dir):
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    try:
        sm = P.ShardedMapping(n_frames, HW, stand_in, own_only=own_only, device="cpu")
        assert (sm.rank, sm.world) == (rank, world)
        params = sm.run()
        torch.save({k: v.clone() for k, v in params.items()}, os.path.join(out_dir, "rank%d.pt" % rank))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("n_frames,own_only", [(7, False), (8, False), (7, True)])
def test_two_ranks_match_the_schedule(tmp_path, n_frames, own_only):
    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), n_frames, own_only, str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    want = schedule_by_hand(n_frames, world, own_only)
    for r in range(world):
        got = torch.load(os.path.join(str(tmp_path), "rank%d.pt" % r))
        assert sorted(got) == list(range(n_frames))
        for i in range(n_frames):
            assert torch.equal(got[i], want[i]), (r, i)


def test_schedule_properties():
    assert P.waves(7, 2) == [[0, 1], [2, 3], [4, 5], [6]]
    assert P.waves(3, 8) == [[0, 1, 2]]
    assert P.neighbours(0) == [] and P.neighbours(2) == [0, 1] and P.neighbours(9) == [5, 6, 7, 8]
    # world 1 is the sequential mapping: every earlier neighbour is fixed
    seq = schedule_by_hand(6, 1, False)
    assert torch.equal(seq[5], stand_in(5, {j: seq[j] for j in range(5)}))
    # with 2 ranks the partner frame of the same wave is not seen
    two = schedule_by_hand(6, 2, False)
    assert torch.equal(two[5], stand_in(5, {j: two[j] for j in range(4)}))
    assert not torch.equal(two[5], seq[5])


def test_single_process_without_a_process_group():
    sm = P.ShardedMapping(5, HW, stand_in, device="cpu")
    assert (sm.rank, sm.world) == (0, 1)
    got = sm.run()
    want = schedule_by_hand(5, 1, False)
    assert all(torch.equal(got[i], want[i]) for i in range(5))
    assert len(sm.wave_s) == 5


def test_one_view_schedule():
    its = [P.view_of_iteration(t, 4) for t in range(100)]
    assert its.count(0) == 40                       # the frame's own view on 40 % of iterations
    assert sorted(set(its)) == [0, 1, 2, 3, 4]
    assert [its.count(k) for k in (1, 2, 3, 4)] == [15, 15, 15, 15]
    assert all(P.view_of_iteration(t, 0) == 0 for t in range(20))
    assert [P.view_of_iteration(t, 2) for t in range(10)] == [0, 0, 1, 2, 1, 0, 0, 2, 1, 2]
