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
* Per-frame memory admission: frames are charged their device footprint
  until their results are home; one that does not fit the frame budget is
  refused with LSAS_ERR_CAPACITY (single or batch submission), or waits for
  room when a wait time is set.
* The learned form: a configuration registered with refinement parameters
  runs LS -> tensor-core refinement -> MRC, and each of its frames, served in
  a mix with plain frames, equals that chain run on the frame alone.
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


def _frame_buffers(c, eq=False):
    import torch
    H = torch.empty((c.M, c.N), dtype=torch.complex64).pin_memory()
    bits = torch.empty(c.D * c.N * c.q // 8, dtype=torch.uint8).pin_memory()
    z = torch.empty((c.D, c.N), dtype=torch.complex64).pin_memory() if eq else None
    return H, bits, z


def test_frames_admitted_by_memory_budget(L):
    """Per-frame admission: each frame is charged its device footprint
    (input + H + bits, + z when asked) until its results are home; a frame
    that does not fit the frame budget is refused (or, with a wait time,
    admitted once earlier frames complete)."""
    c = sweep_config(16, 256)
    b = synth.generate(c, frame_ids=range(3))
    in_b, h_b, bit_b, eq_b = L.frame_bytes(c.M, c.N, c.cp, c.S, c.Q, c.fmt)
    fb = in_b + h_b + bit_b
    # a long batch window keeps the first frames queued on the host
    srv = L.Server(mem_budget=1 << 30, max_batch=16, max_wait_us=2e6)
    cid = srv.register(c.M, c.N, c.cp, c.S, c.pilot_idx, c.Q, fmt=c.fmt, pilot=b.pilot)
    assert srv.frame_bytes()["budget"] == (1 << 30) - srv.stats()["admitted_bytes"]
    # registration admits the plan's own device memory (tables and the
    # split-tail scratch) on top of both lanes' staging for 16 frames
    plan = L.Plan(c.M, c.N, c.cp, c.S, c.pilot_idx, c.Q, fmt=c.fmt, max_frames=16)
    assert srv.stats()["admitted_bytes"] >= plan.device_bytes() + 2 * 16 * (fb + eq_b)
    plan.close()
    srv.set_admission(int(2.5 * fb), 0.0)
    assert srv.frame_bytes() == {"charged": 0, "budget": int(2.5 * fb)}
    xs = [_pinned(b.frames[f]) for f in range(3)]
    outs = [_frame_buffers(c) for _ in range(3)]
    t0 = srv.submit(cid, xs[0], *outs[0][:2])
    t1 = srv.submit(cid, xs[1], *outs[1][:2])
    assert srv.frame_bytes()["charged"] == 2 * fb
    with pytest.raises(L.LsasError) as e:
        srv.submit(cid, xs[2], *outs[2][:2])             # a third frame does not fit
    assert e.value.code == L.LSAS_ERR_CAPACITY
    with pytest.raises(L.LsasError) as e:
        srv.submit_many([(cid, xs[2], *outs[2][:2])])    # nor as a batch: nothing queued
    assert e.value.code == L.LSAS_ERR_CAPACITY
    assert srv.frame_bytes()["charged"] == 2 * fb
    srv.wait(t0)
    srv.wait(t1)
    assert srv.frame_bytes()["charged"] == 0              # released when results are home
    t2 = srv.submit(cid, xs[2], *outs[2][:2])
    srv.wait(t2)
    srv.set_admission(fb // 2, 0.0)                      # a frame larger than the budget
    with pytest.raises(L.LsasError) as e:
        srv.submit(cid, xs[0], *outs[0][:2])
    assert e.value.code == L.LSAS_ERR_CAPACITY
    assert srv.close() == L.LSAS_OK
    # with a wait time, a frame that does not fit yet waits for room
    srv = L.Server(mem_budget=1 << 30, max_batch=1, max_wait_us=0.0)
    cid = srv.register(c.M, c.N, c.cp, c.S, c.pilot_idx, c.Q, fmt=c.fmt, pilot=b.pilot)
    srv.set_admission(int(1.5 * (fb + eq_b)), 10000.0)
    outs = [_frame_buffers(c, eq=True) for _ in range(3)]
    tickets = [srv.submit(cid, xs[f], *outs[f]) for f in range(3)]
    srv.wait_many(tickets)
    assert srv.frame_bytes()["charged"] == 0 and srv.stats()["frames"] == 3
    assert srv.close() == L.LSAS_OK
    plan = L.Plan(c.M, c.N, c.cp, c.S, c.pilot_idx, c.Q, fmt=c.fmt, max_frames=3, pilot=b.pilot)
    import torch
    Ha, ba, za = plan.run_frame(torch.from_numpy(np.ascontiguousarray(b.frames)).cuda(), want_eq=True)
    plan.sync()
    for f in range(3):
        assert np.array_equal(outs[f][1].numpy(), ba[f].cpu().numpy())
        assert np.array_equal(outs[f][2].numpy().view(np.uint32), za[f].cpu().numpy().view(np.uint32))


def test_learned_form_served_in_a_mix(L):
    """A configuration registered with refinement parameters runs LS ->
    tensor-core refinement -> MRC; its frames, interleaved with plain frames
    of another configuration, equal bit for bit lsas_estimate ->
    lsas_dn_apply_tc -> lsas_demodulate run on each frame alone."""
    import torch
    import paper_1901_07499_gb300.denoiser as D
    dn = D.Denoiser(D.init_params(3) * np.float32(4.0))
    pb = dn.bf16_params()
    cr = sweep_config(16, 512).replace(Q=16)
    cp_ = sweep_config(8, 256)
    F = 5
    br = synth.generate(cr, frame_ids=range(F))
    bp = synth.generate(cp_, frame_ids=range(F))
    srv = L.Server(mem_budget=2 << 30, max_batch=3, max_wait_us=150.0)
    rid = srv.register(cr.M, cr.N, cr.cp, cr.S, cr.pilot_idx, cr.Q, fmt=cr.fmt, pilot=br.pilot,
                       refine_params_bf16=pb)
    pid = srv.register(cp_.M, cp_.N, cp_.cp, cp_.S, cp_.pilot_idx, cp_.Q, fmt=cp_.fmt, pilot=bp.pilot)
    outs_r = [_frame_buffers(cr, eq=True) for _ in range(F)]
    outs_p = [_frame_buffers(cp_) for _ in range(F)]
    tickets = []
    for f in range(F):
        tickets.append(srv.submit(rid, _pinned(br.frames[f]), *outs_r[f]))
        tickets.append(srv.submit(pid, _pinned(bp.frames[f]), *outs_p[f][:2]))
    srv.wait_many(tickets)
    assert srv.close() == L.LSAS_OK
    plan = L.Plan(cr.M, cr.N, cr.cp, cr.S, cr.pilot_idx, cr.Q, fmt=cr.fmt, max_frames=1, pilot=br.pilot)
    for f in range(F):
        x = torch.from_numpy(np.ascontiguousarray(br.frames[f:f + 1])).cuda()
        Hls = plan.estimate(x)
        Hr = dn.apply(Hls, params_bf16=pb, tensor_cores=True)
        bits, eq = plan.demodulate(x, Hr, want_eq=True)
        assert plan.sync_status() == L.LSAS_OK and int(dn.status().item()) == 0
        H, bits_s, eq_s = outs_r[f]
        assert np.array_equal(H.numpy().view(np.uint32), Hr[0].cpu().numpy().view(np.uint32))
        assert np.array_equal(bits_s.numpy(), bits[0].cpu().numpy())
        assert np.array_equal(eq_s.numpy().view(np.uint32), eq[0].cpu().numpy().view(np.uint32))
    plan = L.Plan(cp_.M, cp_.N, cp_.cp, cp_.S, cp_.pilot_idx, cp_.Q, fmt=cp_.fmt, max_frames=F,
                  pilot=bp.pilot)
    Ha, ba, _ = plan.run_frame(torch.from_numpy(np.ascontiguousarray(bp.frames)).cuda())
    plan.sync()
    for f in range(F):
        assert np.array_equal(outs_p[f][1].numpy(), ba[f].cpu().numpy())
