"""Multi-rank host logic on CPU with the gloo backend (world size 2).

* bench.py: each rank owns disjoint seeded frames, the reported time is the
  slowest rank's, and the job value counts every rank's samples (weak
  scaling).
* The antenna split across ranks: gather_partials stacks every rank's shard
  partials in rank order, and adding them in that order gives the whole
  array's combined symbols (shard partials from the oracle, on CPU).
"""

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


def _split_worker(rank, world, port, out):
    """Rank r owns antennas [r*M/world, (r+1)*M/world) of oracle frames; the
    gathered partials, added in rank order, give the whole array's z."""
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import numpy as np
    import torch
    import torch.distributed as dist
    import oracle
    import synth
    from synth.frames import sweep_config
    from paper_1901_07499_gb300.lsas import gather_partials
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}",
                            rank=rank, world_size=world)
    cfg = sweep_config(6, 64)
    b = synth.generate(cfg, frame_ids=range(2))
    ref = oracle.receive(b.frames, cfg.N, cfg.cp, cfg.S, cfg.pilot_idx, cfg.Q, b.pilot)
    ds = oracle.data_symbols(cfg.S, cfg.pilot_idx)
    a, c = rank * cfg.M // world, (rank + 1) * cfg.M // world
    P = np.stack([oracle.mrc_partial(ref.H[f, a:c], ref.Y[f, a:c][:, ds])[0] for f in range(2)])
    E = np.stack([oracle.channel_energy(ref.H[f, a:c]) for f in range(2)])
    Pt = torch.from_numpy(P.astype(np.complex64))
    Et = torch.from_numpy(E.astype(np.float32))
    Pa, Ea = gather_partials(Pt, Et)
    assert tuple(Pa.shape) == (world, 2, cfg.D, cfg.N) and tuple(Ea.shape) == (world, 2, cfg.N)
    assert torch.equal(Pa[rank], Pt) and torch.equal(Ea[rank], Et)
    z = np.stack([oracle.mrc_combine(list(Pa[:, f].numpy().astype(np.complex128)),
                                     list(Ea[:, f].numpy().astype(np.float64)))[0]
                  for f in range(2)])
    out[rank] = float(np.max(np.abs(z - ref.z)) / np.sqrt(np.mean(np.abs(ref.z) ** 2)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_antenna_split_gathers_in_rank_order():
    from paper_1901_07499_gb300.build import build
    build()   # once, before the ranks import the binding
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_split_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] < 1e-6 and res[1] < 1e-6
