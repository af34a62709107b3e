"""The benchmark's multi-rank logic on CPU ranks (gloo, world size 2): the job's time and
its capacity flag are the maximum over ranks, and a rank that overflowed makes every rank
see the failure."""
import os
import socket

import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out_dir):
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    try:
        t = bench.max_over_ranks(10.0 + 5.0 * rank, world, "cpu")            # per-rank step times
        ok = bench.max_over_ranks(0.0 if rank == 0 else 1.0, world, "cpu") == 0.0   # rank 1 overflowed
        with open(os.path.join(out_dir, "r%d" % rank), "w") as f:
            f.write("%r %r" % (t, ok))
    finally:
        dist.destroy_process_group()


def test_max_over_two_gloo_ranks(tmp_path):
    mp.start_processes(_worker, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    for r in range(2):
        assert open(os.path.join(str(tmp_path), "r%d" % r)).read() == "15.0 False"


def test_single_rank_is_the_identity():
    assert bench.max_over_ranks(3.25, 1, "cpu") == 3.25
