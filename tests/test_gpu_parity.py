"""GPU parity: the CUDA library (through its C ABI) against the FP64 oracle
on the same seeded synthetic frames.

Covers the whole path (lsas_run_frame), each step alone (lsas_fft = CP
removal + FFT, lsas_estimate = LS, lsas_demodulate = MRC + demap with the
oracle's channel), the antenna-count x FFT-length grid, odd shapes (M not a
multiple of the antennas per block, M = 1, M = 256, one data symbol,
CP = N - 1, pilot not first, the two-symbol kernel's step pairings and
group layers, the paper's CP 72, a CP that defeats the bulk-copy alignment, BPSK and 256-QAM, float32
input), full-scale amplitudes, the zero-energy status, argument errors,
the host-buffer entry point, determinism, and the 1000-frame 64-antenna
N=1024 workload in the launch configuration the benchmark times (device
resident, and from pinned host memory as the end-to-end leg runs it).
"""

import numpy as np
import pytest

import oracle
import synth
from synth.frames import FrameConfig, sweep_config, paper_config
from tests.parity_util import (check_frame_outputs, oracle_run, rel_err,
                               to_torch_frames, unpack, TOL_REL)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import torch
    assert torch.cuda.is_available()
    import paper_1901_07499_gb300.lsas as lsas
    return lsas


def make_plan(L, cfg, max_frames=1024):
    return L.Plan(cfg.M, cfg.N, cfg.cp, cfg.S, cfg.pilot_idx, cfg.Q, fmt=cfg.fmt,
                  max_frames=max_frames, pilot=synth.frames.pilot_sequence(cfg))


def run_and_check(L, cfg, F=None, want_eq=True, pilot=None, split=True):
    import torch
    ids = range(F if F is not None else cfg.F)
    b = synth.generate(cfg, frame_ids=ids, pilot=pilot)
    plan = make_plan(L, cfg)
    if pilot is not None:
        plan.set_pilot(pilot)
    if not split:
        plan.set_batch_split(False)
    x = to_torch_frames(b)
    H, bits, eq = plan.run_frame(x, want_eq=want_eq)
    plan.sync()
    ref = oracle_run(cfg, b)
    return check_frame_outputs(cfg, ref, H.cpu().numpy(), bits.cpu().numpy(),
                               eq.cpu().numpy() if eq is not None else None), plan


def test_tiny_config_full(L):
    cfg = synth.CONFIGS["tiny"]
    stats, plan = run_and_check(L, cfg)
    assert plan.info()["tma"] == 1


def test_scale_config_small_batch(L):
    run_and_check(L, synth.CONFIGS["scale"], F=3)


def test_precision_config_small_batch(L):
    run_and_check(L, synth.CONFIGS["precision"], F=2)


@pytest.mark.parametrize("M", [8, 16, 32, 64, 128])
@pytest.mark.parametrize("N", [64, 256, 512, 1024, 2048])
def test_sweep_grid(L, M, N):
    run_and_check(L, sweep_config(M, N), F=2)


@pytest.mark.parametrize("N", [128])
@pytest.mark.parametrize("M", [1, 3, 13, 100])
def test_odd_antenna_counts(L, M, N):
    run_and_check(L, sweep_config(M, N).replace(M=M), F=3)


@pytest.mark.parametrize("M", [2, 3, 5, 13])
def test_odd_antenna_counts_n2048(L, M):
    """N = 2048 from sc16 rows runs four warp pairs per frame, antenna m on
    pair m mod 4: fewer antennas than pairs, and a last round that leaves
    some pairs idle."""
    run_and_check(L, sweep_config(16, 2048).replace(M=M), F=2)


def test_single_antenna_n2048(L):
    """M = 1: MRC is single-antenna zero forcing, z = Y / H.  Near a deep fade
    (the seeded channel has a subcarrier at 5e-5 of the mean power) the
    float32 error of Y and H is divided by |H_k|, so the plain 1e-4 bar on z
    does not follow from the arithmetic there.  H keeps the 1e-4 bar; z is
    held to the error that the 1e-4 bars on Y and H imply through z = Y / H:
    |dz_k| <= 1e-4 (rms(Y) + |z_k| rms(H)) / |H_k|; bits as everywhere."""
    import torch
    cfg = sweep_config(16, 2048).replace(M=1)
    b = synth.generate(cfg, frame_ids=range(2))
    plan = make_plan(L, cfg)
    H, bits, eq = plan.run_frame(to_torch_frames(b), want_eq=True)
    plan.sync()
    ref = oracle_run(cfg, b, keep_Y=True)
    check_frame_outputs(cfg, ref, H.cpu().numpy(), bits.cpu().numpy(), None)
    z = eq.cpu().numpy()
    rmsY = np.sqrt(np.mean(np.abs(ref.Y) ** 2, axis=(1, 2, 3)))[:, None, None]
    rmsH = np.sqrt(np.mean(np.abs(ref.H) ** 2, axis=(1, 2)))[:, None, None]
    Hk = np.abs(ref.H[:, 0, :])[:, None, :]
    bound = TOL_REL * (rmsY + np.abs(ref.z) * rmsH) / Hk
    assert np.all(np.abs(z - ref.z) <= bound)
    same_prec, _ = oracle.demap(z.astype(np.complex64), cfg.Q, dtype=np.float32)
    q = int(round(np.log2(cfg.Q)))
    assert np.array_equal(same_prec, unpack(bits.cpu().numpy(), cfg.D, cfg.N, q))


@pytest.mark.parametrize("M,N", [(16, 64), (16, 1024), (5, 1024)])
def test_paper_shapes(L, M, N):
    run_and_check(L, paper_config(M, N, F=2))


@pytest.mark.parametrize("M,N,F", [(256, 256, 2), (256, 1024, 1), (256, 2048, 1)])
def test_maximum_antenna_count(L, M, N, F):
    """M = 256, the largest the interface takes, on the per-warp (N <= 1024) and
    warp-pair (N = 2048) fused kernels."""
    run_and_check(L, sweep_config(M, N).replace(M=M), F=F)


@pytest.mark.parametrize("N,S", [(256, 2), (1024, 2), (2048, 3)])
def test_fewest_symbols(L, N, S):
    """One pilot and one (or two) data symbols: a single data-symbol group."""
    run_and_check(L, sweep_config(16, N).replace(S=S), F=3)


@pytest.mark.parametrize("M,S,pilot_idx", [
    (1, 2, 0), (9, 3, 2), (13, 4, 0), (64, 5, 4), (16, 6, 3), (24, 9, 0), (40, 14, 7),
    (72, 17, 16)])
def test_two_symbol_kernel_groupings(L, M, S, pilot_idx):
    """N = 1024 from aligned sc16 rows runs the two-symbol kernel, whose steps
    pair up the rows of a data-symbol group (the pilot with the first three
    data symbols, then four at a time): odd item counts leave a step with one
    row, a data symbol beside the pilot or alone accumulates on its own
    columns and the others interleaved in pairs; idle warps (M < 8, M not a
    multiple of 8), one to sixteen data symbols, the pilot anywhere."""
    run_and_check(L, sweep_config(M, 1024).replace(S=S, pilot_idx=pilot_idx), F=2)


@pytest.mark.parametrize("M,N,S,pilot_idx", [
    (32, 512, 14, 0), (37, 512, 5, 4), (71, 512, 17, 16), (40, 512, 2, 1),
    (128, 256, 14, 0), (131, 256, 9, 3), (158, 256, 4, 0)])
def test_two_symbol_kernel_antenna_teams(L, M, N, S, pilot_idx):
    """N = 512 with 32 or more antennas and N = 256 with 128 or more run the
    two-symbol kernel with 2 or 4 antennas per warp step (lane teams of 16 or
    8 lanes, a radix-16 or radix-8 second pass): ragged antenna counts leave
    teams of the last step idle, with the step pairings of every group."""
    run_and_check(L, sweep_config(M, N).replace(S=S, pilot_idx=pilot_idx), F=2)


@pytest.mark.parametrize("M,S,pilot_idx", [
    (1, 2, 0), (5, 3, 2), (4, 4, 0), (13, 5, 4), (8, 9, 0), (20, 14, 7), (9, 17, 16)])
def test_two_symbol_pair_kernel_groupings(L, M, S, pilot_idx):
    """N = 2048 from aligned sc16 rows runs the two-symbol pair kernel, with
    the same step pairings as at N = 1024: odd item counts, a data symbol
    beside the pilot or alone, idle pairs (M < 4, M not a multiple of 4),
    one to sixteen data symbols, the pilot anywhere."""
    run_and_check(L, sweep_config(M, 2048).replace(S=S, pilot_idx=pilot_idx), F=2)


@pytest.mark.parametrize("N,S,pilot_idx", [(1024, 17, 5), (1024, 6, 0), (2048, 17, 16), (2048, 5, 2),
                                             (512, 11, 10)])
def test_two_symbol_kernel_group_layers(L, N, S, pilot_idx):
    """Both two-symbol kernels: the one-launch antenna split of a small batch
    gives every data-symbol group its own block (each transforms the pilot,
    group 0 alone writes H and the energy): against the oracle, and H equal
    to the unsplit call's."""
    import torch
    cfg = sweep_config(40 if N == 512 else 16, N).replace(S=S, pilot_idx=pilot_idx)
    F, G = 2, 2
    b = synth.generate(cfg, frame_ids=range(F))
    plan = make_plan(L, cfg, max_frames=4)
    x = to_torch_frames(b)
    H, bits, eq = plan.empty_H(F), plan.empty_bits(F), plan.empty_eq(F)
    st = L.lsas_run_frame_split_static(plan.handle, x.data_ptr(), F, G, H.data_ptr(),
                                       bits.data_ptr(), eq.data_ptr(),
                                       torch.cuda.current_stream().cuda_stream)
    assert st == L.LSAS_OK
    assert plan.sync_status() == L.LSAS_OK
    ref = oracle_run(cfg, b)
    check_frame_outputs(cfg, ref, H.cpu().numpy(), bits.cpu().numpy(), eq.cpu().numpy())
    H1, _, _ = plan.run_frame(x)
    plan.sync()
    assert torch.equal(H, H1)


@pytest.mark.parametrize("N", [64, 1024, 2048])
def test_longest_cyclic_prefix(L, N):
    """CP = N - 1, the largest the interface takes (rows no longer 16-byte
    aligned: the plain-load path)."""
    run_and_check(L, sweep_config(8, N).replace(cp=N - 1), F=2)


@pytest.mark.parametrize("pilot_idx", [1, 6, 13])
def test_pilot_not_first(L, pilot_idx):
    run_and_check(L, sweep_config(24, 512).replace(pilot_idx=pilot_idx), F=2)


@pytest.mark.parametrize("pilot_idx", [4, 13])
def test_pilot_not_first_n2048(L, pilot_idx):
    run_and_check(L, sweep_config(12, 2048).replace(pilot_idx=pilot_idx), F=2)


@pytest.mark.parametrize("split", [True, False])
@pytest.mark.parametrize("N", [256, 1024, 2048])
@pytest.mark.parametrize("Q", [2, 4, 64, 256])
def test_qam_orders(L, Q, N, split):
    """Every constellation through each fused receiver the plan picks at 16
    antennas: the one-symbol kernel (N = 256) and the two-symbol kernels
    (N = 1024, 2048), whose demap has one copy per constellation.  A small
    batch runs split into antenna shards (the combine kernel slices) unless
    the split is off (the fused kernel slices)."""
    run_and_check(L, sweep_config(16, N).replace(Q=Q, snr_db=40.0), F=2, split=split)


@pytest.mark.parametrize("cp", [17, 1, 0])
def test_unaligned_cp_falls_back_to_plain_loads(L, cp):
    cfg = sweep_config(12, 256).replace(cp=cp, taps=min(8, cp + 1))
    stats, plan = run_and_check(L, cfg, F=2)
    assert plan.info()["tma"] == (1 if (cp * 4) % 16 == 0 else 0)


@pytest.mark.parametrize("N", [64, 1024, 2048])
def test_fc32_input(L, N):
    run_and_check(L, sweep_config(10, N).replace(fmt="fc32"), F=2)


def test_complex_pilot(L):
    cfg = sweep_config(8, 256)
    rng = np.random.default_rng(5)
    pilot = np.exp(2j * np.pi * rng.random(256)) * (0.5 + rng.random(256))
    run_and_check(L, cfg, F=2, pilot=pilot)


# ------------------------------------------------------- single steps ----

@pytest.mark.parametrize("N", [64, 128, 256, 512, 1024, 2048])
def test_fft_alone(L, N):
    cfg = sweep_config(9, N).replace(S=5)
    b = synth.generate(cfg, frame_ids=range(2))
    plan = make_plan(L, cfg)
    Y = plan.fft(to_torch_frames(b))
    plan.sync()
    ref = oracle_run(cfg, b, keep_Y=True)
    e = rel_err(Y.cpu().numpy(), ref.Y, axes=(1, 2, 3))
    assert e.max() <= TOL_REL, e


def test_fft_full_scale_amplitudes(L):
    cfg = sweep_config(8, 1024).replace(S=3)
    b = synth.generate(cfg, frame_ids=range(1))
    rng = np.random.default_rng(1)
    b.frames[...] = rng.choice(np.array([-32767, 32767], np.int16), size=b.frames.shape)
    plan = make_plan(L, cfg)
    Y = plan.fft(to_torch_frames(b))
    plan.sync()
    ref = oracle_run(cfg, b, keep_Y=True)
    assert rel_err(Y.cpu().numpy(), ref.Y, axes=(1, 2, 3)).max() <= TOL_REL


@pytest.mark.parametrize("M,N", [(8, 64), (64, 1024), (13, 2048)])
def test_estimate_alone(L, M, N):
    cfg = sweep_config(M, N)
    b = synth.generate(cfg, frame_ids=range(2))
    plan = make_plan(L, cfg)
    H = plan.estimate(to_torch_frames(b))
    plan.sync()
    ref = oracle_run(cfg, b)
    assert rel_err(H.cpu().numpy(), ref.H, axes=(1, 2)).max() <= TOL_REL


@pytest.mark.parametrize("M,N", [(8, 64), (64, 1024), (20, 2048)])
def test_demodulate_with_oracle_channel(L, M, N):
    import torch
    cfg = sweep_config(M, N)
    b = synth.generate(cfg, frame_ids=range(2))
    ref = oracle_run(cfg, b)
    plan = make_plan(L, cfg)
    Hd = torch.from_numpy(ref.H.astype(np.complex64)).cuda()
    bits, eq = plan.demodulate(to_torch_frames(b), Hd, want_eq=True)
    plan.sync()
    check_frame_outputs(cfg, ref, None, bits.cpu().numpy(), eq.cpu().numpy(), check_H=False)


def test_zero_channel_energy_latches_status(L):
    import torch
    cfg = sweep_config(8, 256)
    b = synth.generate(cfg, frame_ids=range(2))
    ref = oracle_run(cfg, b)
    H = ref.H.astype(np.complex64).copy()
    H[1, :, 17] = 0
    plan = make_plan(L, cfg)
    bits, eq = plan.demodulate(to_torch_frames(b), torch.from_numpy(H).cuda(), want_eq=True)
    assert plan.sync_status() == L.LSAS_ERR_DEVICE
    assert plan.sync_status() == L.LSAS_OK          # cleared by the read
    z = eq.cpu().numpy()
    assert np.all(z[1, :, 17] == 0)
    ref2 = oracle_run(cfg, b, H_given=H.astype(np.complex128))
    assert ref2.bad[1] and not ref2.bad[0]
    got = unpack(bits.cpu().numpy(), cfg.D, cfg.N, cfg.q)
    assert np.array_equal(got[1, :, 17], ref2.bits[1, :, 17])


def test_argument_errors(L):
    import ctypes as C
    import torch
    cfg = sweep_config(8, 256)
    plan = make_plan(L, cfg, max_frames=4)
    x = torch.zeros((5, 8, cfg.T, 2), dtype=torch.int16, device="cuda")
    H = plan.empty_H(5)
    bits = plan.empty_bits(5)
    s = torch.cuda.current_stream().cuda_stream
    h = plan.handle
    assert L.lsas_run_frame(h, x.data_ptr(), 5, H.data_ptr(), bits.data_ptr(), None, s) == L.LSAS_ERR_CAPACITY
    assert L.lsas_run_frame(h, x.data_ptr(), 0, H.data_ptr(), bits.data_ptr(), None, s) == L.LSAS_OK
    assert L.lsas_run_frame(h, None, 2, H.data_ptr(), bits.data_ptr(), None, s) == L.LSAS_ERR_INVALID_ARG
    assert L.lsas_run_frame(h, x.data_ptr(), 2, None, bits.data_ptr(), None, s) == L.LSAS_ERR_INVALID_ARG
    assert L.lsas_run_frame(h, x.data_ptr(), -1, H.data_ptr(), bits.data_ptr(), None, s) == L.LSAS_ERR_INVALID_ARG
    bad = np.zeros(2 * 256, np.float32)
    assert L.lsas_plan_set_pilot(h, bad.ctypes.data_as(C.POINTER(C.c_float))) == L.LSAS_ERR_INVALID_ARG
    assert L.lsas_plan_set(h, 7, 4) == L.LSAS_ERR_INVALID_ARG
    out = C.c_void_p()
    assert L.lsas_plan_create(8, 1000, 16, 4, 0, 16, C.byref(out)) == L.LSAS_ERR_INVALID_ARG
    assert out.value is None
    assert plan.sync_status() == L.LSAS_OK


@pytest.mark.parametrize("M,N", [(32, 512), (16, 128)])
def test_host_entry_point_matches_device_path(L, M, N):
    """The host-buffer path (N = 512: prefixes stripped in the transfer;
    N = 128: whole rows) gives the device path's bytes exactly."""
    import torch
    cfg = sweep_config(M, N)
    b = synth.generate(cfg, frame_ids=range(150))   # > 2 transfer chunks
    plan = make_plan(L, cfg)
    xd = to_torch_frames(b)
    H, bits, eq = plan.run_frame(xd, want_eq=True)
    plan.sync()
    xh = torch.from_numpy(b.frames).pin_memory()
    Hh = torch.empty(H.shape, dtype=H.dtype).pin_memory()
    bh = torch.empty(bits.shape, dtype=bits.dtype).pin_memory()
    eh = torch.empty(eq.shape, dtype=eq.dtype).pin_memory()
    plan.run_frame_host(xh, Hh, bh, eh)
    plan.sync()
    assert torch.equal(Hh, H.cpu()) and torch.equal(bh, bits.cpu()) and torch.equal(eh, eq.cpu())
    assert plan.host_input_bytes_per_frame() == cfg.M * cfg.S * (cfg.N if N >= 256 else cfg.N + cfg.cp) * 4


def test_deterministic(L):
    import torch
    cfg = sweep_config(64, 1024)
    b = synth.generate(cfg, frame_ids=range(3))
    plan = make_plan(L, cfg)
    x = to_torch_frames(b)
    r1 = plan.run_frame(x, want_eq=True)
    r2 = plan.run_frame(x, want_eq=True)
    plan.sync()
    assert all(torch.equal(a, c) for a, c in zip(r1, r2))


# ---------------------------------------------------- batch split ----

@pytest.mark.parametrize("name,F", [("scale", 3), ("precision", 2)])
def test_batch_split_small_batch(L, name, F):
    """A batch smaller than one wave runs split into antenna shards (partial
    sums, then the combine pass): split and unsplit both meet the oracle
    bars, and H is the same bytes (each antenna's LS is the same
    arithmetic either way)."""
    import torch
    cfg = synth.CONFIGS[name]
    b = synth.generate(cfg, frame_ids=range(F))
    plan = make_plan(L, cfg, max_frames=8)
    assert plan.batch_split_shards(F) > 1
    x = to_torch_frames(b)
    ref = oracle_run(cfg, b)
    H1, bits1, eq1 = plan.run_frame(x, want_eq=True)
    plan.sync()
    check_frame_outputs(cfg, ref, H1.cpu().numpy(), bits1.cpu().numpy(), eq1.cpu().numpy())
    plan.set_batch_split(False)
    assert plan.batch_split_shards(F) == 1
    H0, bits0, eq0 = plan.run_frame(x, want_eq=True)
    plan.sync()
    check_frame_outputs(cfg, ref, H0.cpu().numpy(), bits0.cpu().numpy(), eq0.cpu().numpy())
    assert torch.equal(H0, H1)
    with pytest.raises(L.LsasError):
        L.check(L.lsas_plan_set_batch_split(plan.handle, 3), "lsas_plan_set_batch_split")
    # one shard count for every batch smaller than a wave: a frame gives the
    # same bytes alone and in a batch
    plan.set_batch_split(2)
    shards = {plan.batch_split_shards(n) for n in range(1, 9)}
    assert len(shards) == 1 and shards.pop() > 1
    H2, bits2, eq2 = plan.run_frame(x, want_eq=True)
    Ha, bitsa, eqa = plan.run_frame(x[:1].contiguous(), want_eq=True)
    plan.sync()
    assert torch.equal(H2[:1], Ha) and torch.equal(bits2[:1], bitsa) and torch.equal(eq2[:1], eqa)
    check_frame_outputs(cfg, ref, H2.cpu().numpy(), bits2.cpu().numpy(), eq2.cpu().numpy())


@pytest.mark.parametrize("N,fmt", [(2048, "fc32"), (512, "sc16")])
def test_batch_split_other_kernels(L, N, fmt):
    """The shard pass of the warp-specialised kernel (N = 2048 from fc32 rows)
    and of the two-symbol kernel with two antennas per warp step (N = 512,
    64 antennas): split and unsplit small batches both meet the oracle bars,
    H equal (the plan picks one kernel for all its launches)."""
    import torch
    cfg = sweep_config(16, N).replace(fmt=fmt, M=64 if N == 512 else 16)
    b = synth.generate(cfg, frame_ids=range(2))
    plan = make_plan(L, cfg, max_frames=4)
    assert plan.batch_split_shards(2) > 1
    x = to_torch_frames(b)
    ref = oracle_run(cfg, b)
    H1, bits1, eq1 = plan.run_frame(x, want_eq=True)
    plan.sync()
    check_frame_outputs(cfg, ref, H1.cpu().numpy(), bits1.cpu().numpy(), eq1.cpu().numpy())
    plan.set_batch_split(False)
    H0, bits0, eq0 = plan.run_frame(x, want_eq=True)
    plan.sync()
    check_frame_outputs(cfg, ref, H0.cpu().numpy(), bits0.cpu().numpy(), eq0.cpu().numpy())
    assert torch.equal(H0, H1)


def test_batch_split_tail_after_whole_wave(L):
    """One whole wave of frames plus two: the wave runs one frame per block,
    the two after it split into antenna shards; every frame meets the
    oracle bars.  Two such calls on one plan from two streams at once take
    turns on the plan's partial-sum array and both stay right."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    cfg = sweep_config(64, 256)
    F = sms + 2
    b = synth.generate(cfg, frame_ids=range(F))
    plan = make_plan(L, cfg, max_frames=F)
    assert plan.batch_split_shards(F) == 2
    assert plan.batch_split_shards(sms) == 1
    ref = oracle_run(cfg, b)
    x = to_torch_frames(b)
    x2 = torch.flip(x, dims=[0]).contiguous()
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    torch.cuda.synchronize()
    outs = []
    for xs, st in zip((x, x2), streams):
        with torch.cuda.stream(st):
            outs.append(plan.run_frame(xs, want_eq=True, stream=st))
    torch.cuda.synchronize()
    assert plan.sync_status() == L.LSAS_OK
    H, bits, eq = (t.cpu().numpy() for t in outs[0])
    check_frame_outputs(cfg, ref, H, bits, eq)
    H2, bits2, eq2 = (t.cpu().numpy() for t in outs[1])
    # the flipped batch: its last two frames (split) are frames 1 and 0
    for f2, f in ((F - 2, 1), (F - 1, 0), (0, F - 1)):
        assert np.array_equal(H2[f2], H[f])
    tail = synth.generate(cfg, frame_ids=[1, 0])
    check_frame_outputs(cfg, oracle_run(cfg, tail), H2[F - 2:], bits2[F - 2:], eq2[F - 2:])


# ------------------------------------------------ full-size workload ----

def test_scale_workload_full_size_sampled(L):
    """1000 frames of 64 antennas x 1024 subcarriers in one launch, the
    configuration the benchmark times: a pool of seeded frames is tiled to
    1000 frames; sampled frames are checked against the oracle, and every
    frame against the first copy of its pool frame."""
    import torch
    cfg = synth.CONFIGS["scale"]
    pool = 8
    b = synth.generate(cfg, frame_ids=range(pool))
    plan = make_plan(L, cfg)
    x = to_torch_frames(b).repeat(cfg.F // pool, 1, 1, 1)
    H, bits, eq = plan.run_frame(x, want_eq=True)
    plan.sync()
    for f in (0, 517, 999):
        p = f % pool
        one = synth.generate(cfg, frame_ids=[p])
        ref = oracle_run(cfg, one)
        check_frame_outputs(cfg, ref, H[f:f + 1].cpu().numpy(), bits[f:f + 1].cpu().numpy(),
                            eq[f:f + 1].cpu().numpy())
    Hr = H.view(cfg.F // pool, pool, cfg.M, cfg.N)
    assert torch.equal(Hr, Hr[:1].expand_as(Hr))
    br = bits.view(cfg.F // pool, pool, -1)
    assert torch.equal(br, br[:1].expand_as(br))


def test_scale_workload_full_size_host_path(L):
    """The end-to-end leg of the benchmark: 1000 frames from pinned host memory
    through lsas_run_frame_host (chunked uploads with the cyclic prefixes
    stripped, kernels, downloads) equal the device-resident call byte for byte,
    and two sampled frames meet the oracle bars."""
    import torch
    cfg = synth.CONFIGS["scale"]
    pool = 8
    b = synth.generate(cfg, frame_ids=range(pool))
    plan = make_plan(L, cfg)
    x = to_torch_frames(b).repeat(cfg.F // pool, 1, 1, 1)
    H, bits, _ = plan.run_frame(x)
    plan.sync()
    xh = x.cpu().pin_memory()
    del x
    Hh = torch.empty(H.shape, dtype=H.dtype).pin_memory()
    bh = torch.empty(bits.shape, dtype=bits.dtype).pin_memory()
    plan.run_frame_host(xh, Hh, bh)
    plan.sync()
    assert torch.equal(Hh, H.cpu()) and torch.equal(bh, bits.cpu())
    for f in (3, 998):
        ref = oracle_run(cfg, synth.generate(cfg, frame_ids=[f % pool]))
        check_frame_outputs(cfg, ref, Hh[f:f + 1].numpy(), bh[f:f + 1].numpy(), None)


@pytest.mark.parametrize("M", [13, 64])
def test_tensor_core_and_cuda_core_fused_kernels(L, M, monkeypatch):
    """N = 1024 with aligned sc16 rows: the default fused kernel (two symbols
    per warp step, both FFT passes on the CUDA cores), with
    LSAS_FUSED_KERNEL=warp the one-symbol-per-step kernel, and with
    LSAS_FUSED_KERNEL=tensor the one whose second pass runs on the tensor
    cores.  All meet the oracle bars on the same frames (full receiver and
    lsas_demodulate with the oracle's channel), including an antenna count
    that leaves some warps without a second antenna (M = 13)."""
    cfg = synth.CONFIGS["scale"].replace(M=M)
    b = synth.generate(cfg, frame_ids=range(3))
    ref = oracle_run(cfg, b)
    ref_d = oracle_run(cfg, b, H_given=ref.H)
    x = to_torch_frames(b)
    import torch
    for kernel in ("tensor", "warp", "default"):
        if kernel == "default":
            monkeypatch.delenv("LSAS_FUSED_KERNEL", raising=False)
        else:
            monkeypatch.setenv("LSAS_FUSED_KERNEL", kernel)
        plan = make_plan(L, cfg, max_frames=4)
        H, bits, eq = plan.run_frame(x, want_eq=True)
        assert plan.sync_status() == L.LSAS_OK
        check_frame_outputs(cfg, ref, H.cpu().numpy(), bits.cpu().numpy(), eq.cpu().numpy())
        Hd = torch.from_numpy(ref.H.astype(np.complex64)).cuda()
        bits_d, eq_d = plan.demodulate(x, Hd, want_eq=True)
        assert plan.sync_status() == L.LSAS_OK
        check_frame_outputs(cfg, ref_d, None, bits_d.cpu().numpy(), eq_d.cpu().numpy(),
                            check_H=False)
        plan.close()
