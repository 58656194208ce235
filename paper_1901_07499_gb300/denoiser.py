"""Learned refinement of the LS channel estimate: parameters, training and
checkpoints around the CUDA kernels of liblsas (lsas_dn_*).

Every numeric step (normalisation, the convolutions, the loss, gradients,
Adam, bf16 rounding) runs in the library's kernels; this module only holds
device buffers and marshals calls.  Training data are LS-domain pairs from
``synth.ls_pairs`` (true channel rows and their LS estimates).

Checkpoint file: the 8-byte magic ``LSASDN01``, then little-endian int64
n_params, step, seed, rows_seen, then float32 params, first moments, second
moments (n_params each).
"""

from __future__ import annotations

import ctypes as C
import struct
from typing import Optional

import numpy as np

from . import lsas as L

MAGIC = b"LSASDN01"


def init_params(seed: int = 0) -> np.ndarray:
    """He-style initial weights, zero biases, a small last layer, so the
    residual network starts close to the identity (plain LS)."""
    rng = np.random.default_rng(seed)
    shapes = [(32, 2, 5), (32,), (32, 32, 5), (32,), (32, 32, 5), (32,), (2, 32, 5), (2,)]
    parts = []
    for i, s in enumerate(shapes):
        if len(s) == 1:
            parts.append(np.zeros(s))
        else:
            parts.append(rng.standard_normal(s) * np.sqrt(2.0 / (s[1] * s[2])) * (0.1 if i == 6 else 1.0))
    p = np.concatenate([x.reshape(-1) for x in parts]).astype(np.float32)
    assert p.size == L.LSAS_DN_PARAMS
    return p


class Denoiser:
    def __init__(self, params: Optional[np.ndarray] = None, seed: int = 0, device="cuda"):
        import torch
        self.device = torch.device(device)
        p = init_params(seed) if params is None else np.asarray(params, np.float32)
        self.params = torch.from_numpy(p.copy()).to(self.device)
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.grad = torch.zeros_like(self.params)
        self.loss = torch.zeros(1, dtype=torch.float32, device=self.device)
        self.step = 0
        self.seed = seed
        self.rows_seen = 0
        self._work = None
        self._work_key = None
        self._status = None

    def work(self, R: int, N: int):
        import torch
        n = C.c_size_t()
        L.check(L.lsas_dn_work_size(R, N, C.byref(n)), "lsas_dn_work_size")
        if self._work is None or self._work.numel() < n.value:
            self._work = torch.empty(n.value, dtype=torch.float32, device=self.device)
        return self._work

    def compute_grad(self, Hls, Ht, tensor_cores: bool = False):
        """Loss and gradient on rows Hls, Ht [R][N] complex64 (device).

        ``tensor_cores``: the BF16 pass on tcgen05 (bf16 operands and stored
        tensors, fp32 sums; the fp32 parameters are rounded to bf16 for it);
        otherwise the FP32 pass on the CUDA cores."""
        R, N = int(Hls.shape[0]), int(Hls.shape[1])
        if tensor_cores:
            L.check(L.lsas_dn_grad_tc(L._ptr(self.params), L._ptr(Hls), L._ptr(Ht), R, N,
                                      L._ptr(self.work(R, N)), L._ptr(self.grad),
                                      L._ptr(self.loss), L._ptr(self.status()), L._stream(None)),
                    "lsas_dn_grad_tc")
        else:
            L.check(L.lsas_dn_grad(L._ptr(self.params), L._ptr(Hls), L._ptr(Ht), R, N,
                                   L._ptr(self.work(R, N)), L._ptr(self.grad), L._ptr(self.loss),
                                   L._stream(None)), "lsas_dn_grad")
        return self.loss, self.grad

    def train_step(self, Hls, Ht, lr: float = 1e-3, tensor_cores: bool = False):
        self.compute_grad(Hls, Ht, tensor_cores=tensor_cores)
        self.step += 1
        L.check(L.lsas_dn_adam(L._ptr(self.params), L._ptr(self.grad), L._ptr(self.m),
                               L._ptr(self.v), self.step, lr, L._stream(None)), "lsas_dn_adam")
        self.rows_seen += int(Hls.shape[0])
        return self.loss

    def bf16_params(self):
        import torch
        q = torch.empty(L.LSAS_DN_PARAMS, dtype=torch.uint16 if hasattr(torch, "uint16") else torch.int16,
                        device=self.device)
        L.check(L.lsas_dn_to_bf16(L._ptr(self.params), L._ptr(q), L._stream(None)), "lsas_dn_to_bf16")
        return q

    def status(self):
        """Device status word of the tensor-core path (0, or 6 after a wait
        that gave up); created on first use."""
        import torch
        if self._status is None:
            self._status = torch.zeros(1, dtype=torch.int32, device=self.device)
        return self._status

    def apply(self, H, out=None, bf16: bool = True, params_bf16=None, tensor_cores: bool = False):
        """Refined rows of H [..., N] complex64 (device; rows = all leading axes).

        ``tensor_cores``: the 32 -> 32 layers on tcgen05 with bf16 activations
        (bf16 parameters only)."""
        import torch
        N = int(H.shape[-1])
        R = int(H.numel() // N)
        if out is None:
            out = torch.empty_like(H)
        if tensor_cores:
            if not bf16:
                raise ValueError("the tensor-core path reads bf16 parameters")
            pb = params_bf16 if params_bf16 is not None else self.bf16_params()
            L.check(L.lsas_dn_apply_tc(L._ptr(pb), L._ptr(H), R, N, L._ptr(self.work(R, N)),
                                       L._ptr(out), L._ptr(self.status()), L._stream(None)),
                    "lsas_dn_apply_tc")
            return out
        p = (params_bf16 if params_bf16 is not None else self.bf16_params()) if bf16 else self.params
        L.check(L.lsas_dn_apply(L._ptr(p), 1 if bf16 else 0, L._ptr(H), R, N,
                                L._ptr(self.work(R, N)), L._ptr(out), L._stream(None)),
                "lsas_dn_apply")
        return out

    # ---- checkpoints
    def save(self, path: str) -> None:
        with open(path, "wb") as fh:
            fh.write(MAGIC)
            fh.write(struct.pack("<4q", L.LSAS_DN_PARAMS, self.step, self.seed, self.rows_seen))
            for t in (self.params, self.m, self.v):
                fh.write(t.detach().cpu().numpy().astype("<f4").tobytes())

    @classmethod
    def load(cls, path: str, device="cuda") -> "Denoiser":
        import torch
        with open(path, "rb") as fh:
            if fh.read(8) != MAGIC:
                raise ValueError(f"{path}: not a denoiser checkpoint")
            n, step, seed, rows = struct.unpack("<4q", fh.read(32))
            if n != L.LSAS_DN_PARAMS:
                raise ValueError(f"{path}: {n} parameters, expected {L.LSAS_DN_PARAMS}")
            arrs = [np.frombuffer(fh.read(4 * n), dtype="<f4").copy() for _ in range(3)]
        d = cls(arrs[0], seed=seed, device=device)
        d.m = torch.from_numpy(arrs[1]).to(d.device)
        d.v = torch.from_numpy(arrs[2]).to(d.device)
        d.step, d.rows_seen = step, rows
        return d


def train(rows: int = 200_000, N: int = 1024, batch: int = 256, epochs: int = 1,
          lr: float = 1e-3, seed: int = 0, chunk: int = 8192, log=None,
          tensor_cores: bool = False) -> Denoiser:
    """Train on LS-domain pairs (SNR U[0, 30] dB, 4..16 taps, 1..3 dB/tap);
    ``tensor_cores`` runs every gradient pass in BF16 on tcgen05."""
    import torch
    import synth
    dn = Denoiser(seed=seed)
    for ep in range(epochs):
        done = 0
        c = 0
        while done < rows:
            n = min(chunk, rows - done)
            H, Hls, _ = synth.ls_pairs(n, N, seed=seed * 1_000_003 + c)
            Ht = torch.from_numpy(H.astype(np.complex64)).to(dn.device)
            Hl = torch.from_numpy(Hls.astype(np.complex64)).to(dn.device)
            perm = torch.randperm(n, generator=torch.Generator().manual_seed(seed + ep * 7919 + c))
            for i in range(0, n - batch + 1, batch):
                idx = perm[i:i + batch].to(dn.device)
                loss = dn.train_step(Hl[idx].contiguous(), Ht[idx].contiguous(), lr,
                                     tensor_cores=tensor_cores)
            if log is not None:
                log(ep, done + n, float(loss.item()))
            done += n
            c += 1
    return dn
