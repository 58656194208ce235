"""Out-of-bounds write checks without a sanitizer: output canaries.

Every device output buffer handed to the library sits in the middle of a
larger allocation whose 4 KB guard regions on both sides are filled with the
byte 0xA5.  After the call (and a synchronise) the guards must still hold
0xA5 everywhere, the buffer itself must have been written, and the inputs
must be unchanged.  Shapes are small, end in partial tiles, and cover every
kernel family: the fused receiver for N = 64..2048 (sc16 and fc32), the
staged estimate / demodulate / FFT path, the antenna split (caller partials
and the static scratch), the tensor-core FFT and receive_y, packet detection
and the fftshift, the learned refinement (apply, tensor-core apply,
gradient, Adam, bf16 rounding), and the host-buffer path (guards in pinned
host memory).  Zero-frame calls of every frame-based entry point return OK
and write nothing.
"""

import numpy as np
import pytest

import synth
from synth.frames import sweep_config

pytestmark = pytest.mark.gpu

GUARD = 4096
FILL = 0xA5


@pytest.fixture(scope="module")
def L():
    import torch
    assert torch.cuda.is_available()
    import paper_1901_07499_gb300.lsas as lsas
    return lsas


class Guarded:
    """A tensor of the given shape and dtype inside a guarded allocation."""

    def __init__(self, shape, dtype, device="cuda", pinned=False):
        import torch
        n = int(np.prod(shape)) * torch.empty((), dtype=dtype).element_size()
        self.nbytes = n
        self.store = torch.full((2 * GUARD + n,), FILL, dtype=torch.uint8, device=device)
        if pinned:
            self.store = self.store.pin_memory()
        self.t = self.store[GUARD:GUARD + n].view(dtype).view(shape)

    def check(self, name):
        import torch
        torch.cuda.synchronize()
        s = self.store.cpu().numpy()
        assert np.all(s[:GUARD] == FILL), f"{name}: write before the buffer"
        assert np.all(s[GUARD + self.nbytes:] == FILL), f"{name}: write past the buffer"
        assert np.any(s[GUARD:GUARD + self.nbytes] != FILL), f"{name}: buffer never written"


def _frames(cfg, F, seed=0):
    import torch
    b = synth.generate(cfg.replace(seed=cfg.seed + seed), frame_ids=range(F))
    return b, torch.from_numpy(np.ascontiguousarray(b.frames)).cuda()


def _plan(L, cfg, F):
    b = synth.generate(cfg, frame_ids=range(1))
    return L.Plan(cfg.M, cfg.N, cfg.cp, cfg.S, cfg.pilot_idx, cfg.Q, fmt=cfg.fmt, max_frames=F,
                  pilot=b.pilot)


def _outs(plan, F, eq=True):
    import torch
    H = Guarded((F, plan.M, plan.N), torch.complex64)
    bits = Guarded((F, plan.D * plan.N * plan.q // 8), torch.uint8)
    z = Guarded((F, plan.D, plan.N), torch.complex64) if eq else None
    return H, bits, z


@pytest.mark.parametrize("M,N,fmt", [(5, 64, "sc16"), (3, 64, "fc32"), (7, 256, "sc16"),
                                     (9, 1024, "sc16"), (3, 2048, "sc16")])
def test_fused_receiver(L, M, N, fmt):
    cfg = sweep_config(M, N).replace(fmt=fmt)
    F = 3
    _, x = _frames(cfg, F)
    x0 = x.clone()
    plan = _plan(L, cfg, F)
    H, bits, z = _outs(plan, F)
    plan.run_frame(x, H.t, bits.t, z.t)
    plan.sync()
    for g, n in ((H, "H"), (bits, "bits"), (z, "eq")):
        g.check(n)
    assert (x == x0).all()


def test_staged_path_and_split(L):
    import torch
    cfg = sweep_config(10, 512)
    F = 2
    _, x = _frames(cfg, F)
    plan = _plan(L, cfg, F)
    H, bits, z = _outs(plan, F)
    plan.estimate(x, H.t)
    plan.demodulate(x, H.t, bits.t, z.t)
    Y = Guarded((F, cfg.M, cfg.S, cfg.N), torch.complex64)
    plan.fft(x, Y.t)
    plan.sync()
    for g, n in ((H, "estimate H"), (bits, "demodulate bits"), (z, "demodulate eq"), (Y, "fft Y")):
        g.check(n)
    # caller partials: three uneven shards
    G = 3
    P = Guarded((G, F, cfg.D, cfg.N), torch.complex64)
    E = Guarded((G, F, cfg.N), torch.float32)
    H2, bits2, z2 = _outs(plan, F)
    m0 = 0
    for g in range(G):
        mc = cfg.M // G + (1 if g < cfg.M % G else 0)
        plan.mrc_partial(x, m0, mc, H2.t, P.t[g], E.t[g])
        m0 += mc
    plan.mrc_combine(P.t, E.t, bits2.t, z2.t)
    plan.sync()
    for g, n in ((P, "partials P"), (E, "partials E"), (H2, "split H"), (bits2, "combine bits"),
                 (z2, "combine eq")):
        g.check(n)
    # the static split: equal shards (one launch) and unequal shards
    for shards in (2, 3):
        H3, bits3, z3 = _outs(plan, F)
        plan.run_frame_split(x, shards, H3.t, bits3.t, z3.t)
        plan.sync()
        for g, n in ((H3, "static split H"), (bits3, "static split bits"), (z3, "static split eq")):
            g.check(f"{n} ({shards} shards)")


def test_tensor_core_fft_and_receive_y(L):
    import torch
    cfg = sweep_config(6, 1024)
    F = 2
    _, x = _frames(cfg, F)
    plan = _plan(L, cfg, F)
    Y = Guarded((F, cfg.M, cfg.S, cfg.N), torch.complex64)
    plan.fft_tc(x, 3, Y.t)
    plan.sync()
    Y.check("fft_tc Y")
    H, bits, z = _outs(plan, F)
    plan.receive_y(Y.t, H.t, bits.t, z.t)
    plan.sync()
    for g, n in ((H, "receive_y H"), (bits, "receive_y bits"), (z, "receive_y eq")):
        g.check(n)


def test_packet_detection_and_shift(L):
    import torch
    cfg = sweep_config(4, 256)
    F, window = 3, 300
    cap = synth.generate_capture(cfg, frame_ids=range(F), max_delay=window)
    c = torch.from_numpy(np.ascontiguousarray(cap.captures)).cuda()
    plan = _plan(L, cfg, F)
    plan.set_pn(synth.pn_sequence())
    off = Guarded((F,), torch.int32)
    peaks = Guarded((F,), torch.float32)
    plan.pn_sync(c, window, off.t, peaks.t)
    plan.sync()
    off.check("pn_sync offsets")
    peaks.check("pn_sync peaks")
    fr = Guarded((F, cfg.M, cfg.S * (cfg.N + cfg.cp), 2), torch.int16)
    plan.pn_extract(c, off.t, 8, fr.t)
    plan.sync()
    fr.check("pn_extract frames")
    H, bits, z = _outs(plan, F)
    plan.run_frame(fr.t, H.t, bits.t, z.t)
    plan.fftshift(L.LSAS_SHIFT_H, H.t)
    plan.fftshift(L.LSAS_SHIFT_EQ, z.t)
    plan.fftshift(L.LSAS_SHIFT_BITS, bits.t)
    plan.sync()
    for g, n in ((H, "shifted H"), (bits, "shifted bits"), (z, "shifted eq")):
        g.check(n)


def test_learned_refinement(L):
    import torch
    import paper_1901_07499_gb300.denoiser as D
    R, N = 5, 384
    Ht, Hls, _ = synth.ls_pairs(R, N, seed=3)
    x = torch.from_numpy(Hls.astype(np.complex64)).cuda()
    t = torch.from_numpy(Ht.astype(np.complex64)).cuda()
    dn = D.Denoiser(D.init_params(1) * np.float32(3.0))
    for bf16, tc in ((False, False), (True, False), (True, True)):
        out = Guarded((R, N), torch.complex64)
        dn.apply(x, out=out.t, bf16=bf16, tensor_cores=tc)
        out.check(f"apply bf16={bf16} tensor_cores={tc}")
    assert int(dn.status().item()) == 0
    # gradient and Adam into guarded parameter-sized buffers
    n = L.LSAS_DN_PARAMS
    grad = Guarded((n,), torch.float32)
    loss = Guarded((1,), torch.float32)
    assert L.lsas_dn_grad(dn.params.data_ptr(), x.data_ptr(), t.data_ptr(), R, N,
                          dn.work(R, N).data_ptr(), grad.t.data_ptr(), loss.t.data_ptr(),
                          torch.cuda.current_stream().cuda_stream) == L.LSAS_OK
    grad.check("grad")
    loss.check("loss")
    p, m, v = (Guarded((n,), torch.float32) for _ in range(3))
    p.t.copy_(dn.params)
    m.t.zero_()
    v.t.zero_()
    assert L.lsas_dn_adam(p.t.data_ptr(), grad.t.data_ptr(), m.t.data_ptr(), v.t.data_ptr(), 1,
                          1e-3, torch.cuda.current_stream().cuda_stream) == L.LSAS_OK
    for g, name in ((p, "adam params"), (m, "adam m"), (v, "adam v")):
        g.check(name)
    q = Guarded((n,), torch.int16)
    assert L.lsas_dn_to_bf16(dn.params.data_ptr(), q.t.data_ptr(),
                             torch.cuda.current_stream().cuda_stream) == L.LSAS_OK
    q.check("bf16 params")


def test_host_buffer_path(L):
    import torch
    cfg = sweep_config(8, 512)
    F = 70                                           # two transfer chunks, the second partial
    b = synth.generate(cfg, frame_ids=range(F))
    plan = _plan(L, cfg, F)
    xh = torch.from_numpy(np.ascontiguousarray(b.frames)).pin_memory()
    H = Guarded((F, cfg.M, cfg.N), torch.complex64, device="cpu", pinned=True)
    bits = Guarded((F, plan.D * cfg.N * plan.q // 8), torch.uint8, device="cpu", pinned=True)
    z = Guarded((F, cfg.D, cfg.N), torch.complex64, device="cpu", pinned=True)
    plan.run_frame_host(xh, H.t, bits.t, z.t)
    plan.sync()
    for g, n in ((H, "host H"), (bits, "host bits"), (z, "host eq")):
        g.check(n)


def test_zero_frames_is_a_no_op(L):
    """Every frame-based entry point accepts n_frames = 0: it returns OK,
    launches nothing and leaves its (guarded) outputs untouched."""
    import torch
    cfg = sweep_config(8, 1024)
    plan = _plan(L, cfg, 4)
    plan.set_pn(synth.pn_sequence())
    s = torch.cuda.current_stream().cuda_stream
    x = torch.zeros((1, cfg.M, cfg.S * (cfg.N + cfg.cp), 2), dtype=torch.int16, device="cuda")
    bufs = {name: Guarded((1 << 16,), torch.uint8) for name in
            ("H", "bits", "eq", "Y", "P", "E", "off", "peak", "frames")}
    pt = {k: v.t.data_ptr() for k, v in bufs.items()}
    h = plan.handle
    calls = {
        "lsas_run_frame": lambda: L.lsas_run_frame(h, x.data_ptr(), 0, pt["H"], pt["bits"], pt["eq"], s),
        "lsas_estimate": lambda: L.lsas_estimate(h, x.data_ptr(), 0, pt["H"], s),
        "lsas_demodulate": lambda: L.lsas_demodulate(h, x.data_ptr(), pt["H"], 0, pt["bits"], pt["eq"], s),
        "lsas_fft": lambda: L.lsas_fft(h, x.data_ptr(), 0, pt["Y"], s),
        "lsas_fft_tc": lambda: L.lsas_fft_tc(h, x.data_ptr(), 0, 3, pt["Y"], s),
        "lsas_receive_y": lambda: L.lsas_receive_y(h, pt["Y"], 0, pt["H"], pt["bits"], pt["eq"], s),
        "lsas_mrc_partial": lambda: L.lsas_mrc_partial(h, x.data_ptr(), 0, 0, cfg.M, pt["H"], pt["P"], pt["E"], s),
        "lsas_mrc_combine": lambda: L.lsas_mrc_combine(h, pt["P"], pt["E"], 2, 0, pt["bits"], pt["eq"], s),
        "lsas_run_frame_split_static": lambda: L.lsas_run_frame_split_static(h, x.data_ptr(), 0, 2, pt["H"],
                                                                             pt["bits"], pt["eq"], s),
        "lsas_pn_sync": lambda: L.lsas_pn_sync(h, x.data_ptr(), 0, 4096, 300, pt["off"], pt["peak"], s),
        "lsas_pn_extract": lambda: L.lsas_pn_extract(h, x.data_ptr(), 0, 4096, pt["off"], 0, pt["frames"], s),
        "lsas_fftshift": lambda: L.lsas_fftshift(h, L.LSAS_SHIFT_H, pt["H"], 0, s),
    }
    for name, call in calls.items():
        assert call() == L.LSAS_OK, name
    plan.sync()
    torch.cuda.synchronize()
    for name, g in bufs.items():
        assert bool((g.store == FILL).all()), f"{name} written by a zero-frame call"
    xh = torch.zeros((1,), dtype=torch.int16).pin_memory()
    assert L.lsas_run_frame_host(h, xh.data_ptr(), 0, pt["H"], pt["bits"], None, s) == L.LSAS_OK
