"""Shared helpers of the GPU parity tests: run the CUDA library and the FP64
oracle on the same seeded frames and compare them with the stated bars.

Bars (per frame): max |H_gpu - H_oracle| / rms(H_oracle) <= 1e-4, the same
for the combined symbols z, and bits identical wherever the oracle's decision
margin is >= 1e-3.  Bits are also compared everywhere against the oracle's
slicer applied to the GPU's own z in float32, the precision the kernel decides
in: that comparison must be exact.
"""

import numpy as np

import oracle

TOL_REL = 1e-4
MARGIN = 1e-3


def rel_err(got, want, axes):
    """max |got - want| / rms(want) over ``axes`` (per leading index)."""
    err = np.max(np.abs(got - want), axis=axes)
    rms = np.sqrt(np.mean(np.abs(want) ** 2, axis=axes))
    return err / np.maximum(rms, 1e-300)


def unpack(bits_bytes, D, N, q):
    F = bits_bytes.shape[0]
    b = np.unpackbits(bits_bytes, axis=-1, bitorder="big")
    return b[:, :D * N * q].reshape(F, D, N, q)


def to_torch_frames(batch, device="cuda"):
    import torch
    return torch.from_numpy(np.ascontiguousarray(batch.frames)).to(device)


def oracle_run(cfg, batch, H_given=None, keep_Y=False):
    return oracle.receive(batch.frames, cfg.N, cfg.cp, cfg.S, cfg.pilot_idx, cfg.Q,
                          batch.pilot, H_given=H_given, keep_Y=keep_Y)


def check_frame_outputs(cfg, ref, H_gpu, bits_gpu, z_gpu, check_H=True):
    """Assert the parity bars; returns a dict of the worst errors."""
    out = {}
    if check_H:
        eH = rel_err(H_gpu, ref.H, axes=(1, 2))
        out["H"] = float(eH.max())
        assert eH.max() <= TOL_REL, f"H rel err {eH.max():.3g}"
    if z_gpu is not None:
        ez = rel_err(z_gpu, ref.z, axes=(1, 2))
        out["z"] = float(ez.max())
        assert ez.max() <= TOL_REL, f"z rel err {ez.max():.3g}"
    q = int(round(np.log2(cfg.Q)))
    got = unpack(bits_gpu, cfg.D, cfg.N, q)
    sure = ref.margin >= MARGIN
    mism = np.any(got != ref.bits, axis=-1) & sure
    out["bit_mismatch"] = int(mism.sum())
    out["excluded"] = int((~sure).sum())
    assert not mism.any(), f"{mism.sum()} symbols differ with margin >= {MARGIN}"
    if z_gpu is not None:
        same_prec, _ = oracle.demap(z_gpu.astype(np.complex64), cfg.Q, dtype=np.float32)
        assert np.array_equal(same_prec, got), "kernel slicer differs from float32 decision"
    return out
