"""Multi-rank logic of bench.py on CPU with the gloo backend (world size 2):
each rank owns disjoint seeded frames, the reported time is the slowest
rank's, and the job value counts every rank's samples (weak scaling)."""

import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import torch.distributed as dist
    import bench
    import synth
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}",
                            rank=rank, world_size=world)
    ids = list(bench.rank_frame_ids(rank, 4))
    t = bench.max_over_ranks(10.0 + rank, world, "cpu")
    cfg = synth.CONFIGS["scale"]
    out[rank] = (ids, t, bench.job_samples(world, 1000, cfg))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_sharding_and_timing():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    ids0, t0, s0 = res[0]
    ids1, t1, s1 = res[1]
    assert set(ids0).isdisjoint(ids1) and len(ids0) == len(ids1) == 4
    assert t0 == t1 == 11.0                       # slowest rank wins
    assert s0 == s1 == 2 * 1000 * 64 * 14 * 1024  # whole-job samples
