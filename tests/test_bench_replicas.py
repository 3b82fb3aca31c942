"""The multi-rank form of bench.py on CPU: two `gloo` ranks, as torchrun would
start them.  The per-frame path does not shard, so N GPUs run N replicas that
render disjoint views; the only cross-rank steps are a barrier and the MAX of
the ranks' times.  These tests cover that host logic without a GPU."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

WORLD = 2


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _view_key(view):
    cam, t = view
    return np.asarray(cam.world_to_cam, np.float32).tobytes() + np.float32(t).tobytes()


def _rank(rank, port, steps):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=WORLD)
    try:
        import bench
        # the job's time is the slowest replica's
        assert bench.max_over_ranks(dist, 10.0 + 2.5 * rank, "cpu") == 12.5
        assert bench.max_over_ranks(dist, 7.0 - rank, "cpu") == 7.0
        # replicas render disjoint views that interleave into the one-GPU sequence
        mine = [_view_key(bench.views(s, rank, WORLD)) for s in range(steps)]
        every = [None] * WORLD
        dist.all_gather_object(every, mine)
        if rank == 0:
            single = [_view_key(bench.views(i, 0, 1)) for i in range(WORLD * steps)]
            merged = [every[i % WORLD][i // WORLD] for i in range(WORLD * steps)]
            assert merged == single
            assert not set(every[0]) & set(every[1])
    finally:
        dist.destroy_process_group()


def test_two_gloo_replicas_take_the_max_time_and_split_the_views():
    mp.spawn(_rank, args=(_free_port(), 60), nprocs=WORLD, join=True)


def test_one_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(None, 3.25, "cpu") == 3.25
