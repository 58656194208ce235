"""Precision report of the tensor-core FFT next to the FP32 path (GPU).

For a workload (default: the precision workload, 128 antennas, N = 2048,
64-QAM, 30 dB) it runs, on the same seeded frames,
  fused    lsas_run_frame (the FP32 hot path)
  fp32     lsas_fft -> lsas_receive_y (staged, FP32 FFT)
  tc3      lsas_fft_tc(terms=3) -> lsas_receive_y (split fp16 operands)
  tc1      lsas_fft_tc(terms=1) -> lsas_receive_y (plain fp16 operands)
and prints one JSON line per variant: max |Y - Y_oracle| / rms (per frame,
worst frame), the same for z, EVM of z against the transmitted symbols next
to the FP64 oracle's EVM, bit mismatches where the oracle's margin is
>= 1e-3, and the device time per frame of the FFT step (or of the whole
fused call) over a tiled batch.

    python tests/report_tc_precision.py [--config precision] [--frames 2] [--timing-frames 64]
    python tests/report_tc_precision.py --profile-only   # one tensor-core FFT launch, for ncu
"""

import argparse
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402
from tests.parity_util import MARGIN, rel_err, unpack  # noqa: E402


def evm_db(z, X):
    return float(10 * np.log10(np.sum(np.abs(z - X) ** 2) / np.sum(np.abs(X) ** 2)))


def device_ms(fn, reps=5):
    import torch
    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--config", default="precision")
    ap.add_argument("--frames", type=int, default=2)
    ap.add_argument("--timing-frames", type=int, default=64)
    ap.add_argument("--profile-only", action="store_true")
    args = ap.parse_args()
    import torch
    import paper_1901_07499_gb300.lsas as lsas

    cfg = synth.config_by_name(args.config)
    if args.profile_only:
        b = synth.generate(cfg, frame_ids=range(4))
        plan = lsas.Plan(cfg.M, cfg.N, cfg.cp, cfg.S, cfg.pilot_idx, cfg.Q, fmt=cfg.fmt,
                         max_frames=16, pilot=b.pilot)
        x = torch.from_numpy(b.frames).cuda().repeat(4, 1, 1, 1).contiguous()
        for _ in range(3):
            plan.fft_tc(x, terms=3)
        plan.sync()
        print("profile run done")
        return

    b = synth.generate(cfg, frame_ids=range(args.frames))
    plan = lsas.Plan(cfg.M, cfg.N, cfg.cp, cfg.S, cfg.pilot_idx, cfg.Q, fmt=cfg.fmt,
                     max_frames=max(args.frames, args.timing_frames), pilot=b.pilot)
    x = torch.from_numpy(np.ascontiguousarray(b.frames)).cuda()
    ref = oracle.receive(b.frames, cfg.N, cfg.cp, cfg.S, cfg.pilot_idx, cfg.Q, b.pilot)
    ds = oracle.data_symbols(cfg.S, cfg.pilot_idx)
    X = b.X[:, ds, :]
    evm_ref = evm_db(ref.z, X)
    sure = ref.margin >= MARGIN

    reps = (args.timing_frames + args.frames - 1) // args.frames
    xt = x.repeat(reps, 1, 1, 1)[:args.timing_frames].contiguous()
    Yt = torch.empty((args.timing_frames, cfg.M, cfg.S, cfg.N), dtype=torch.complex64, device="cuda")
    Ht, bt = plan.empty_H(args.timing_frames), plan.empty_bits(args.timing_frames)

    variants = {
        "fused": (None, lambda: plan.run_frame(xt, Ht, bt)),
        "fp32": (lambda: plan.fft(x), lambda: plan.fft(xt, Y=Yt)),
        "tc3": (lambda: plan.fft_tc(x, terms=3), lambda: plan.fft_tc(xt, terms=3, Y=Yt)),
        "tc1": (lambda: plan.fft_tc(x, terms=1), lambda: plan.fft_tc(xt, terms=1, Y=Yt)),
    }
    for name, (fft, timed) in variants.items():
        out = {"variant": name, "workload": cfg.name, "frames": args.frames,
               "M": cfg.M, "N": cfg.N, "qam": cfg.Q, "snr_db": cfg.snr_db}
        if fft is None:
            H, bits, eq = plan.run_frame(x, want_eq=True)
            out["err_Y"] = None
        else:
            Y = fft()
            plan.sync()
            Yo = oracle.dft(oracle.strip_cp(oracle.to_complex(b.frames[0]), cfg.N, cfg.cp, cfg.S))
            out["err_Y"] = float(rel_err(Y[:1].cpu().numpy(), Yo[None], axes=(1, 2, 3)).max())
            H, bits, eq = plan.receive_y(Y, want_eq=True)
        plan.sync()
        z = eq.cpu().numpy()
        out["err_H"] = float(rel_err(H.cpu().numpy(), ref.H, axes=(1, 2)).max())
        out["err_z"] = float(rel_err(z, ref.z, axes=(1, 2)).max())
        out["evm_db"] = evm_db(z, X)
        out["evm_oracle_db"] = evm_ref
        out["evm_delta_db"] = out["evm_db"] - evm_ref
        got = unpack(bits.cpu().numpy(), cfg.D, cfg.N, cfg.q)
        out["bit_mismatch_where_sure"] = int((np.any(got != ref.bits, axis=-1) & sure).sum())
        ms = device_ms(timed)
        out["timing_frames"] = args.timing_frames
        out["us_per_frame"] = 1e3 * ms / args.timing_frames
        out["timed"] = "lsas_run_frame (whole path)" if fft is None else "FFT step only"
        print(json.dumps(out))


if __name__ == "__main__":
    main()
