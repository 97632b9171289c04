"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): each rank solves its own
scene, the timed region is the slowest rank's, the job rate sums the ranks' work, and the
reference arm runs on rank 0 only."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, r, local = bench.dist_env()
    ms = 10.0 + 5.0 * r                      # rank 1 is the slowest
    slowest = bench.max_over_ranks(ms, dist, "cpu")
    out[rank] = (w, r, bench.scene_seed(r), slowest, bench.job_rate(100, slowest, w))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_gloo():
    mgr = mp.Manager()
    out = mgr.dict()
    port = _free_port()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    (w0, r0, s0, m0, v0), (w1, r1, s1, m1, v1) = out[0], out[1]
    assert (w0, w1, r0, r1) == (2, 2, 0, 1)
    assert s0 != s1                           # independent scenes
    assert m0 == m1 == 15.0                   # max over ranks
    assert v0 == v1 == pytest.approx(2 * 100 / 0.015)


def test_reference_arm_other_ranks_do_nothing(capsys):
    import argparse

    import bench
    bench.run_reference(argparse.Namespace(steps=1, warmup=0), world=2, rank=1)
    assert capsys.readouterr().out == ""
