"""GPU tests of the serving loop (lsas_server_*): frames of three receiver
configurations (different antenna counts, FFT lengths and QAM orders)
submitted interleaved in random order from pinned host memory.

* Every frame's H, bits and z equal, bit for bit, those of the same frame
  run alone through lsas_run_frame (the result does not depend on the mix),
  and meet the oracle bars.
* Admission: a configuration that does not fit the memory budget is refused
  with LSAS_ERR_CAPACITY; an unknown ticket is refused; a wait with no time
  left on a frame still queued behind a long batch window times out and the
  ticket stays valid.
* Batching under load: with no batch window at all (max_wait_us = 0), a burst
  of 64 frames of one configuration still runs in a handful of full batches,
  because a configuration has at most two batches (lanes) in flight and its
  frames accumulate meanwhile; every frame equals its run alone.
* Batch submission: lsas_server_submit_many queues all frames or none (one
  bad entry refuses the call), lsas_server_wait_many returns every frame's
  latency, and the results equal those of single submissions.
"""

import numpy as np
import pytest

import synth
from synth.frames import sweep_config
from tests.parity_util import check_frame_outputs, oracle_run

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import torch
    assert torch.cuda.is_available()
    import paper_1901_07499_gb300.lsas as lsas
    return lsas


def _pinned(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).pin_memory()


def test_mixed_configurations_match_alone(L):
    import torch
    cfgs = [sweep_config(16, 256).replace(Q=4), sweep_config(64, 1024),
            sweep_config(8, 2048).replace(Q=64)]
    F = 5
    batches = [synth.generate(c, frame_ids=range(F)) for c in cfgs]
    srv = L.Server(mem_budget=4 << 30, max_batch=4, max_wait_us=300.0)
    ids = [srv.register(c.M, c.N, c.cp, c.S, c.pilot_idx, c.Q, fmt=c.fmt, pilot=b.pilot)
           for c, b in zip(cfgs, batches)]
    order = [(ci, f) for ci in range(len(cfgs)) for f in range(F)]
    rng = np.random.default_rng(3)
    rng.shuffle(order)
    outs = {}
    tickets = []
    for ci, f in order:
        c = cfgs[ci]
        x = _pinned(batches[ci].frames[f])
        H = torch.empty((c.M, c.N), dtype=torch.complex64).pin_memory()
        bits = torch.empty(c.D * c.N * c.q // 8, dtype=torch.uint8).pin_memory()
        eq = torch.empty((c.D, c.N), dtype=torch.complex64).pin_memory()
        tickets.append(srv.submit(ids[ci], x, H, bits, eq))
        outs[(ci, f)] = (H, bits, eq)
    lat = [srv.wait(t) for t in tickets]
    st = srv.stats()
    assert st["frames"] == len(order) and st["configs"] == 3
    assert 1 <= st["launches"] <= len(order)
    assert min(lat) > 0
    assert srv.close() == L.LSAS_OK
    for ci, c in enumerate(cfgs):
        b = batches[ci]
        plan = L.Plan(c.M, c.N, c.cp, c.S, c.pilot_idx, c.Q, fmt=c.fmt, max_frames=F, pilot=b.pilot)
        ref = oracle_run(c, b)
        Hs, Bs, Zs = [], [], []
        for f in range(F):
            xa = torch.from_numpy(np.ascontiguousarray(b.frames[f:f + 1])).cuda()
            Ha, ba, za = plan.run_frame(xa, want_eq=True)
            plan.sync()
            H, bits, eq = outs[(ci, f)]
            assert np.array_equal(H.numpy().view(np.uint32), Ha[0].cpu().numpy().view(np.uint32))
            assert np.array_equal(bits.numpy(), ba[0].cpu().numpy())
            assert np.array_equal(eq.numpy().view(np.uint32), za[0].cpu().numpy().view(np.uint32))
            Hs.append(H.numpy()); Bs.append(bits.numpy()); Zs.append(eq.numpy())
        check_frame_outputs(c, ref, np.stack(Hs), np.stack(Bs), np.stack(Zs))


def test_admission_tickets_and_timeouts(L):
    import torch
    c = sweep_config(64, 1024)
    srv = L.Server(mem_budget=64 << 20, max_batch=32, max_wait_us=2e6)
    with pytest.raises(L.LsasError) as e:
        srv.register(c.M, c.N, c.cp, c.S, c.pilot_idx, c.Q)   # 32 frames of 4 MB do not fit
    assert e.value.code == L.LSAS_ERR_CAPACITY
    small = sweep_config(8, 256)
    cid = srv.register(small.M, small.N, small.cp, small.S, small.pilot_idx, small.Q)
    assert L.lsas_server_wait(srv.handle, 12345, 1.0, None) == L.LSAS_ERR_INVALID_ARG
    b = synth.generate(small, frame_ids=range(1))
    x = _pinned(b.frames[0])
    H = torch.empty((small.M, small.N), dtype=torch.complex64).pin_memory()
    bits = torch.empty(small.D * small.N * small.q // 8, dtype=torch.uint8).pin_memory()
    t = srv.submit(cid, x, H, bits)
    # one frame waits up to 2 s for 31 more: no results after 1 ms
    assert L.lsas_server_wait(srv.handle, t, 1.0, None) == L.LSAS_ERR_TIMEOUT
    assert srv.wait(t) > 0            # still valid; the batch window closes
    assert srv.close() == L.LSAS_OK


def test_burst_fills_batches_while_lanes_are_busy(L):
    import torch
    c = sweep_config(64, 1024)
    F, B = 64, 8
    b = synth.generate(c, frame_ids=range(4))
    srv = L.Server(mem_budget=2 << 30, max_batch=B, max_wait_us=0.0)
    cid = srv.register(c.M, c.N, c.cp, c.S, c.pilot_idx, c.Q, fmt=c.fmt, pilot=b.pilot)
    xs = [_pinned(b.frames[i]) for i in range(4)]
    outs = [(torch.empty((c.M, c.N), dtype=torch.complex64).pin_memory(),
             torch.empty(c.D * c.N * c.q // 8, dtype=torch.uint8).pin_memory()) for _ in range(F)]
    tickets = [srv.submit(cid, xs[f % 4], *outs[f]) for f in range(F)]   # one burst
    for t in tickets:
        srv.wait(t)
    st = srv.stats()
    assert st["frames"] == F
    assert st["launches"] <= 24, st          # one launch per frame without the lanes
    assert srv.close() == L.LSAS_OK
    plan = L.Plan(c.M, c.N, c.cp, c.S, c.pilot_idx, c.Q, fmt=c.fmt, max_frames=4, pilot=b.pilot)
    Ha, ba, _ = plan.run_frame(torch.from_numpy(np.ascontiguousarray(b.frames)).cuda())
    plan.sync()
    Ha, ba = Ha.cpu().numpy(), ba.cpu().numpy()
    for f, (H, bits) in enumerate(outs):
        assert np.array_equal(H.numpy().view(np.uint32), Ha[f % 4].view(np.uint32))
        assert np.array_equal(bits.numpy(), ba[f % 4])


def test_submit_many_and_wait_many(L):
    import ctypes as C
    import torch
    c = sweep_config(16, 512)
    F = 12
    b = synth.generate(c, frame_ids=range(F))
    srv = L.Server(mem_budget=1 << 30, max_batch=8, max_wait_us=100.0)
    cid = srv.register(c.M, c.N, c.cp, c.S, c.pilot_idx, c.Q, fmt=c.fmt, pilot=b.pilot)
    xs = [_pinned(b.frames[f]) for f in range(F)]
    outs = [(torch.empty((c.M, c.N), dtype=torch.complex64).pin_memory(),
             torch.empty(c.D * c.N * c.q // 8, dtype=torch.uint8).pin_memory()) for _ in range(F)]
    # one bad entry (unknown configuration): nothing is queued
    n = 2
    cids = (C.c_int * n)(cid, cid + 7)
    ptr = lambda t: t.data_ptr()
    arr = lambda vals: (C.c_void_p * n)(*vals)
    tk = (C.c_uint64 * n)()
    assert L.lsas_server_submit_many(srv.handle, n, cids, arr([ptr(xs[0])] * 2), arr([ptr(outs[0][0])] * 2),
                                     arr([ptr(outs[0][1])] * 2), None, tk) == L.LSAS_ERR_INVALID_ARG
    assert srv.stats()["frames"] == 0
    tickets = srv.submit_many([(cid, xs[f], *outs[f]) for f in range(F)])
    assert len(tickets) == F and len(set(tickets)) == F
    lat = srv.wait_many(tickets)
    assert len(lat) == F and min(lat) > 0
    assert srv.stats()["frames"] == F
    assert srv.close() == L.LSAS_OK
    plan = L.Plan(c.M, c.N, c.cp, c.S, c.pilot_idx, c.Q, fmt=c.fmt, max_frames=F, pilot=b.pilot)
    Ha, ba, _ = plan.run_frame(torch.from_numpy(np.ascontiguousarray(b.frames)).cuda())
    plan.sync()
    for f in range(F):
        assert np.array_equal(outs[f][0].numpy().view(np.uint32), Ha[f].cpu().numpy().view(np.uint32))
        assert np.array_equal(outs[f][1].numpy(), ba[f].cpu().numpy())
