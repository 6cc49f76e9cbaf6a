"""Multi-GPU runs are replicas (frames are independent): the only
cross-rank step is the bench's timing aggregation.  Checked here with two
gloo ranks on the CPU."""
import os
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, ws, port, q):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    slow = bench.max_over_ranks(torch, 1.5 + rank, ws, device="cpu")   # rank 1 is slower
    fps = bench.job_frames_per_s(8 * 10, ws, slow)
    q.put((rank, slow, fps))
    dist.destroy_process_group()


def test_two_rank_aggregation_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, slow, fps in got:
        assert slow == pytest.approx(2.5)                 # the slowest rank decides
        assert fps == pytest.approx(160 / 2.5)            # all frames of both replicas


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(torch, 3.25, 1) == 3.25
    assert bench.job_frames_per_s(8, 1, 2.0) == 4.0
