"""lsas_run_frame_split_static: the antenna-split receiver with its partial
sums in the library's fixed device scratch (no allocation in the call).

Called through the C ABI and compared with the allocating entry points on
the same frames: lsas_mrc_partial + lsas_mrc_combine over caller-allocated
partials (same shards, same order: identical bits, eq within 1e-6 of its
rms) and lsas_run_frame.  Equal shards run as one launch with a grid row per
shard (N = 2048 included); the other cases launch once per shard.  Two calls in a row must both match, and the
second must leave the device's free memory unchanged.  Sizes beyond the
scratch are refused with LSAS_ERR_CAPACITY.  The file name keeps it last in collection;
it also passes alone in a fresh process.
"""

import numpy as np
import pytest

import synth
from synth.frames import sweep_config
from tests.parity_util import MARGIN, check_frame_outputs, oracle_run, unpack

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import torch
    assert torch.cuda.is_available()
    import paper_1901_07499_gb300.lsas as lsas
    return lsas


def _plan(L, cfg):
    return L.Plan(cfg.M, cfg.N, cfg.cp, cfg.S, cfg.pilot_idx, cfg.Q, fmt=cfg.fmt,
                  max_frames=64, pilot=synth.frames.pilot_sequence(cfg))


def _split_allocating(L, plan, x, G):
    """The same split with caller-allocated partials."""
    import torch
    F = x.shape[0]
    H = plan.empty_H(F)
    P, E = plan.empty_partials(F, G)
    m0 = 0
    for g in range(G):
        mc = plan.M // G + (1 if g < plan.M % G else 0)
        plan.mrc_partial(x, m0, mc, H, P[g], E[g])
        m0 += mc
    bits, eq = plan.mrc_combine(P, E, want_eq=True)
    torch.cuda.synchronize()
    return H, bits, eq


@pytest.mark.parametrize("M,N,G,F", [(8, 64, 2, 4), (13, 1024, 3, 3), (64, 1024, 4, 2),
                                     (64, 1024, 8, 1), (16, 256, 16, 2), (32, 2048, 4, 1),
                                     (12, 2048, 5, 2)])
def test_static_split_matches_allocating_path(L, M, N, G, F):
    import torch
    cfg = sweep_config(M, N).replace(M=M)
    b = synth.generate(cfg, frame_ids=range(F))
    plan = _plan(L, cfg)
    x = torch.from_numpy(np.ascontiguousarray(b.frames)).cuda()
    H_ref, bits_ref, eq_ref = _split_allocating(L, plan, x, G)
    H1, bits1, _ = plan.run_frame(x)
    H = plan.empty_H(F)
    bits = plan.empty_bits(F)
    eq = plan.empty_eq(F)
    s = torch.cuda.current_stream().cuda_stream
    free = []
    for call in range(2):
        H.zero_()
        bits.zero_()
        eq.zero_()
        torch.cuda.synchronize()
        before = torch.cuda.mem_get_info()[0]
        st = L.lsas_run_frame_split_static(plan.handle, x.data_ptr(), F, G, H.data_ptr(),
                                           bits.data_ptr(), eq.data_ptr(), s)
        assert st == L.LSAS_OK, L.lsas_status_str(st)
        assert plan.sync_status() == L.LSAS_OK
        # free device memory around the call (the first call of a process may
        # load the library's module, which holds the scratch)
        free.append((before, torch.cuda.mem_get_info()[0]))
        assert torch.equal(H, H_ref) and torch.equal(H, H1)
        assert torch.equal(bits, bits_ref)
        e = eq.cpu().numpy()
        r = eq_ref.cpu().numpy()
        assert np.max(np.abs(e - r)) <= 1e-6 * np.sqrt(np.mean(np.abs(r) ** 2))
        # and the unsharded fused receiver, wherever the oracle is sure
        ref = oracle_run(cfg, b)
        got = unpack(bits.cpu().numpy(), cfg.D, cfg.N, cfg.q)
        want = unpack(bits1.cpu().numpy(), cfg.D, cfg.N, cfg.q)
        assert not np.any(np.any(got != want, axis=-1) & (ref.margin >= MARGIN))
        check_frame_outputs(cfg, ref, H.cpu().numpy(), bits.cpu().numpy(), e)
    assert free[1][1] == free[1][0]


def test_static_split_refuses_sizes_beyond_scratch(L):
    import torch
    cfg = synth.CONFIGS["scale"]
    plan = _plan(L, cfg)
    per = cfg.D * cfg.N * 8 + cfg.N * 4
    limit = L.LSAS_STATIC_SCRATCH_BYTES // per          # shard-frames that fit: 151
    assert limit == 151
    x = torch.zeros((38, cfg.M, cfg.T, 2), dtype=torch.int16, device="cuda")
    H = plan.empty_H(38)
    bits = plan.empty_bits(38)
    s = torch.cuda.current_stream().cuda_stream
    call = lambda F, G: L.lsas_run_frame_split_static(
        plan.handle, x.data_ptr(), F, G, H.data_ptr(), bits.data_ptr(), None, s)
    assert call(38, 4) == L.LSAS_ERR_CAPACITY       # 152 shard-frames
    assert call(76, 2) == L.LSAS_ERR_CAPACITY
    assert call(1, 0) == L.LSAS_ERR_INVALID_ARG
    assert call(1, cfg.M + 1) == L.LSAS_ERR_INVALID_ARG
    assert call(0, 4) == L.LSAS_OK
    assert L.lsas_run_frame_split_static(plan.handle, None, 1, 1, H.data_ptr(),
                                         bits.data_ptr(), None, s) == L.LSAS_ERR_INVALID_ARG
    # a misaligned eq buffer is refused before the shard pass runs: H keeps
    # its sentinel
    eq = torch.zeros(2 * cfg.D * cfg.N * 2 + 4, dtype=torch.float32, device="cuda")
    H.fill_(7.0)
    torch.cuda.synchronize()
    assert L.lsas_run_frame_split_static(plan.handle, x.data_ptr(), 1, 4, H.data_ptr(),
                                         bits.data_ptr(), eq.data_ptr() + 4, s) == L.LSAS_ERR_INVALID_ARG
    torch.cuda.synchronize()
    assert bool((H == 7.0).all())
    assert plan.sync_status() == L.LSAS_OK
