"""GPU parity of packet detection (lsas_pn_sync), frame extraction
(lsas_pn_extract) and the fftshift output order (lsas_fftshift) against the
FP64 oracle on seeded captures with a PN preamble.

* The detected preamble start equals the oracle's argmax wherever the
  oracle's peak is clear of the runner-up, lies on one of the channel's paths
  (delay <= offset < delay + taps), and the peak power matches the oracle's
  metric there.
* Frames cut out after the detected preamble (backoff into the CP) and run
  through the fused receiver meet the usual bars against the oracle run on
  the frames it cuts out itself; the bits are the transmitted ones wherever
  the oracle is sure.
* fftshift of H, z, Y and packed bits equals numpy's fftshift; twice is the
  identity.
* A start outside the capture zero-fills and latches LSAS_ERR_DEVICE;
  argument errors are refused.
"""

import numpy as np
import pytest

import oracle
import synth
from synth.frames import FrameConfig
from tests.parity_util import MARGIN, check_frame_outputs, unpack

pytestmark = pytest.mark.gpu

CFGS = [
    FrameConfig(M=8, N=256, cp=32, S=6, Q=16, taps=4, decay_db=2.0, snr_db=15.0, fmt="sc16",
                name="capture-small"),
    FrameConfig(M=64, N=1024, cp=128, S=14, Q=16, taps=8, decay_db=2.0, snr_db=(10.0, 30.0),
                fmt="sc16", name="capture-scale"),
    FrameConfig(M=4, N=64, cp=16, S=4, Q=4, taps=3, decay_db=3.0, snr_db=20.0, fmt="fc32",
                name="capture-fc32"),
]


@pytest.fixture(scope="module")
def L():
    import torch
    assert torch.cuda.is_available()
    import paper_1901_07499_gb300.lsas as lsas
    return lsas


def make_plan(L, cfg, F):
    plan = L.Plan(cfg.M, cfg.N, cfg.cp, cfg.S, cfg.pilot_idx, cfg.Q, fmt=cfg.fmt,
                  max_frames=max(F, 8), pilot=synth.frames.pilot_sequence(cfg))
    plan.set_pn(synth.pn_sequence())
    return plan


@pytest.mark.parametrize("cfg", CFGS, ids=lambda c: c.name)
def test_pn_sync_and_extracted_receive(L, cfg):
    import torch
    F, max_delay = 4, 400
    c = synth.generate_capture(cfg, frame_ids=range(F), max_delay=max_delay)
    plan = make_plan(L, cfg, F)
    cap = torch.from_numpy(np.ascontiguousarray(c.captures)).cuda()
    offs, peaks = plan.pn_sync(cap, max_delay)
    plan.sync()
    offs, peaks = offs.cpu().numpy(), peaks.cpu().numpy()
    backoff = cfg.cp // 4
    T = cfg.S * (cfg.N + cfg.cp)
    for f in range(F):
        y = oracle.to_complex(c.captures[f])
        o_off, metric = oracle.pn_sync(y, c.pn, max_delay)
        second = np.max(np.delete(metric, o_off))
        if metric[o_off] > second * (1 + 1e-3):
            assert offs[f] == o_off
        assert c.delay[f] <= offs[f] < c.delay[f] + cfg.taps
        assert abs(peaks[f] - metric[offs[f]]) <= 1e-4 * metric[offs[f]]
    frames = plan.pn_extract(cap, torch.from_numpy(offs).cuda(), backoff=backoff)
    H, bits, eq = plan.run_frame(frames, want_eq=True)
    plan.sync()
    ofr = np.stack([oracle.extract_frame(c.captures[f], offs[f] + 255 - backoff, T)
                    for f in range(F)])
    assert np.array_equal(frames.cpu().numpy(), ofr)
    ref = oracle.receive(ofr, cfg.N, cfg.cp, cfg.S, cfg.pilot_idx, cfg.Q, c.pilot)
    check_frame_outputs(cfg, ref, H.cpu().numpy(), bits.cpu().numpy(), eq.cpu().numpy())
    got = unpack(bits.cpu().numpy(), cfg.D, cfg.N, cfg.q)
    sure = ref.margin >= MARGIN
    # at these SNRs the combined symbols decide the transmitted bits where sure
    assert np.mean(np.any(got != c.bits, axis=-1)[sure]) < 1e-3


def test_fftshift_outputs(L):
    import torch
    cfg = CFGS[0]
    b = synth.generate(cfg.replace(snr_db=25.0), frame_ids=range(3))
    plan = make_plan(L, cfg, 3)
    x = torch.from_numpy(np.ascontiguousarray(b.frames)).cuda()
    H, bits, eq = plan.run_frame(x, want_eq=True)
    Y = plan.fft(x)
    plan.sync()
    H0, b0, z0, Y0 = H.cpu().numpy(), bits.cpu().numpy(), eq.cpu().numpy(), Y.cpu().numpy()
    plan.fftshift(L.LSAS_SHIFT_H, H)
    plan.fftshift(L.LSAS_SHIFT_EQ, eq)
    plan.fftshift(L.LSAS_SHIFT_Y, Y)
    plan.fftshift(L.LSAS_SHIFT_BITS, bits)
    plan.sync()
    assert np.array_equal(H.cpu().numpy(), oracle.fftshift_rows(H0))
    assert np.array_equal(eq.cpu().numpy(), oracle.fftshift_rows(z0))
    assert np.array_equal(Y.cpu().numpy(), oracle.fftshift_rows(Y0))
    u0 = unpack(b0, cfg.D, cfg.N, cfg.q)
    u1 = unpack(bits.cpu().numpy(), cfg.D, cfg.N, cfg.q)
    assert np.array_equal(u1, np.fft.fftshift(u0, axes=2))
    plan.fftshift(L.LSAS_SHIFT_H, H)
    plan.fftshift(L.LSAS_SHIFT_BITS, bits)
    plan.sync()
    assert np.array_equal(H.cpu().numpy(), H0) and np.array_equal(bits.cpu().numpy(), b0)


def test_sync_refusals_and_out_of_range(L):
    import torch
    cfg = CFGS[0]
    s = torch.cuda.current_stream().cuda_stream
    plan = L.Plan(cfg.M, cfg.N, cfg.cp, cfg.S, cfg.pilot_idx, cfg.Q, fmt=cfg.fmt, max_frames=2)
    Lc = 300 + 255 + cfg.S * (cfg.N + cfg.cp)
    cap = torch.zeros((2, cfg.M, Lc, 2), dtype=torch.int16, device="cuda")
    offs = torch.zeros(2, dtype=torch.int32, device="cuda")
    bad, ok = L.LSAS_ERR_INVALID_ARG, L.LSAS_OK
    assert L.lsas_pn_sync(plan.handle, cap.data_ptr(), 2, Lc, 100, offs.data_ptr(), None, s) == bad
    plan.set_pn(synth.pn_sequence())
    assert L.lsas_pn_sync(plan.handle, cap.data_ptr(), 2, Lc, Lc - 253, offs.data_ptr(), None, s) == bad
    assert L.lsas_pn_sync(plan.handle, cap.data_ptr(), 2, Lc, Lc - 254, offs.data_ptr(), None, s) == ok
    assert L.lsas_pn_sync(plan.handle, cap.data_ptr(), 3, Lc, 10, offs.data_ptr(), None, s) == L.LSAS_ERR_CAPACITY
    assert L.lsas_fftshift(plan.handle, 7, offs.data_ptr(), 1, s) == bad
    assert L.lsas_pn_extract(plan.handle, cap.data_ptr(), 2, Lc, offs.data_ptr(), -1, cap.data_ptr(), s) == bad
    assert plan.sync_status() == ok
    # a start past the end of the capture
    far = torch.full((2,), Lc, dtype=torch.int32, device="cuda")
    fr = plan.pn_extract(cap + 1, far, backoff=0)
    assert plan.sync_status() == L.LSAS_ERR_DEVICE
    assert int(fr.abs().max()) == 0
