"""ctypes binding of liblsas (include/lsas.h).

Argument marshalling only: every step of the receiver runs in the CUDA
library.  The raw entry points are exposed under their C names
(``lsas_plan_create``, ``lsas_estimate`` ...); :class:`Plan` wraps them for
PyTorch tensors, which supply device memory and streams.  Importing this
module fails loudly when the library has not been built: there is no other
implementation to fall back to.
"""

from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

from .build import LIB

if not os.path.exists(LIB):
    raise ImportError(
        f"liblsas is not built ({LIB} missing); run "
        "`python -c 'import __graft_entry__ as g; g.build()'` first")

_lib = C.CDLL(LIB)

LSAS_OK = 0
LSAS_ERR_INVALID_ARG = 1
LSAS_ERR_UNSUPPORTED = 2
LSAS_ERR_OOM = 3
LSAS_ERR_CAPACITY = 4
LSAS_ERR_CUDA = 5
LSAS_ERR_TIMEOUT = 6
LSAS_ERR_DEVICE = 7
LSAS_STATIC_SCRATCH_BYTES = 16 << 20
LSAS_SHIFT_H, LSAS_SHIFT_EQ, LSAS_SHIFT_Y, LSAS_SHIFT_BITS = 0, 1, 2, 3
LSAS_DN_PARAMS = 10978
LSAS_IN_SC16 = 0
LSAS_IN_FC32 = 1

_vp, _i, _f = C.c_void_p, C.c_int, C.c_float


def _proto(name, args, res=C.c_int):
    fn = getattr(_lib, name)
    fn.argtypes = args
    fn.restype = res
    return fn


lsas_status_str = _proto("lsas_status_str", [_i], C.c_char_p)
lsas_check_config = _proto("lsas_check_config", [_i] * 6)
lsas_frame_bytes = _proto("lsas_frame_bytes", [_i] * 6 + [C.POINTER(C.c_size_t)])
lsas_plan_create = _proto("lsas_plan_create", [_i] * 6 + [C.POINTER(_vp)])
lsas_plan_set = _proto("lsas_plan_set", [_vp, _i, _i])
lsas_plan_set_pilot = _proto("lsas_plan_set_pilot", [_vp, C.POINTER(_f)])
lsas_fft = _proto("lsas_fft", [_vp, _vp, _i, _vp, _vp])
lsas_estimate = _proto("lsas_estimate", [_vp, _vp, _i, _vp, _vp])
lsas_demodulate = _proto("lsas_demodulate", [_vp, _vp, _vp, _i, _vp, _vp, _vp])
lsas_run_frame = _proto("lsas_run_frame", [_vp, _vp, _i, _vp, _vp, _vp, _vp])
lsas_run_frame_host = _proto("lsas_run_frame_host", [_vp, _vp, _i, _vp, _vp, _vp, _vp])
lsas_mrc_partial = _proto("lsas_mrc_partial", [_vp, _vp, _i, _i, _i, _vp, _vp, _vp, _vp])
lsas_mrc_combine = _proto("lsas_mrc_combine", [_vp, _vp, _vp, _i, _i, _vp, _vp, _vp])
lsas_run_frame_split_static = _proto("lsas_run_frame_split_static",
                                     [_vp, _vp, _i, _i, _vp, _vp, _vp, _vp])
lsas_fft_tc = _proto("lsas_fft_tc", [_vp, _vp, _i, _i, _vp, _vp])
lsas_fft_tc_ex = _proto("lsas_fft_tc_ex", [_vp, _vp, _i, _i, _i, _vp, _vp])
LSAS_TC_FP16, LSAS_TC_BF16 = 0, 1
lsas_receive_y = _proto("lsas_receive_y", [_vp, _vp, _i, _vp, _vp, _vp, _vp])
lsas_plan_set_pn = _proto("lsas_plan_set_pn", [_vp, C.POINTER(_f), _i])
lsas_pn_sync = _proto("lsas_pn_sync", [_vp, _vp, _i, _i, _i, _vp, _vp, _vp])
lsas_pn_extract = _proto("lsas_pn_extract", [_vp, _vp, _i, _i, _vp, _i, _vp, _vp])
lsas_fftshift = _proto("lsas_fftshift", [_vp, _i, _vp, _i, _vp])
lsas_server_create = _proto("lsas_server_create", [C.c_size_t, _i, C.c_double, C.POINTER(_vp)])
lsas_server_register = _proto("lsas_server_register",
                              [_vp, _i, _i, _i, _i, _i, _i, _i, C.POINTER(_f), C.POINTER(_i)])
lsas_server_submit = _proto("lsas_server_submit",
                            [_vp, _i, _vp, _vp, _vp, _vp, C.POINTER(C.c_uint64)])
lsas_server_wait = _proto("lsas_server_wait", [_vp, C.c_uint64, C.c_double, C.POINTER(C.c_double)])
lsas_server_stats = _proto("lsas_server_stats", [_vp, C.POINTER(C.c_uint64)])
lsas_server_submit_many = _proto("lsas_server_submit_many",
                                 [_vp, _i, C.POINTER(_i), C.POINTER(_vp), C.POINTER(_vp),
                                  C.POINTER(_vp), C.POINTER(_vp), C.POINTER(C.c_uint64)])
lsas_server_wait_many = _proto("lsas_server_wait_many",
                               [_vp, _i, C.POINTER(C.c_uint64), C.c_double, C.POINTER(C.c_double),
                                C.POINTER(_i)])
lsas_server_destroy = _proto("lsas_server_destroy", [_vp])
lsas_server_register_refined = _proto("lsas_server_register_refined",
                                      [_vp, _i, _i, _i, _i, _i, _i, _i, C.POINTER(_f), _vp,
                                       C.POINTER(_i)])
lsas_server_set_admission = _proto("lsas_server_set_admission", [_vp, C.c_size_t, C.c_double])
lsas_server_frame_bytes = _proto("lsas_server_frame_bytes", [_vp, C.POINTER(C.c_uint64)])
lsas_dn_work_size = _proto("lsas_dn_work_size", [_i, _i, C.POINTER(C.c_size_t)])
lsas_dn_apply = _proto("lsas_dn_apply", [_vp, _i, _vp, _i, _i, _vp, _vp, _vp])
lsas_dn_grad = _proto("lsas_dn_grad", [_vp, _vp, _vp, _i, _i, _vp, _vp, _vp, _vp])
lsas_dn_adam = _proto("lsas_dn_adam", [_vp, _vp, _vp, _vp, _i, C.c_float, _vp])
lsas_dn_to_bf16 = _proto("lsas_dn_to_bf16", [_vp, _vp, _vp])
lsas_dn_apply_tc = _proto("lsas_dn_apply_tc", [_vp, _vp, _i, _i, _vp, _vp, _vp, _vp])
lsas_dn_grad_tc = _proto("lsas_dn_grad_tc", [_vp, _vp, _vp, _i, _i, _vp, _vp, _vp, _vp, _vp])
lsas_plan_set_fault = _proto("lsas_plan_set_fault", [_vp, _i])
lsas_plan_set_batch_split = _proto("lsas_plan_set_batch_split", [_vp, _i])
lsas_plan_batch_split_shards = _proto("lsas_plan_batch_split_shards", [_vp, _i, C.POINTER(_i)])
lsas_run_frame_refined = _proto("lsas_run_frame_refined",
                                [_vp, _vp, _i, _vp, _vp, _vp, _vp, _vp, _vp, _vp])
lsas_plan_set_profile = _proto("lsas_plan_set_profile", [_vp, _i])
lsas_plan_profile = _proto("lsas_plan_profile", [_vp, C.c_char_p, C.c_size_t, C.POINTER(C.c_size_t)])
lsas_plan_sync = _proto("lsas_plan_sync", [_vp, _vp])
lsas_plan_info = _proto("lsas_plan_info", [_vp, C.POINTER(_i)])
lsas_plan_device_bytes = _proto("lsas_plan_device_bytes", [_vp, C.POINTER(C.c_size_t)])
lsas_plan_destroy = _proto("lsas_plan_destroy", [_vp])
lsas_fma_peak_run = _proto("lsas_fma_peak_run", [_i, _i, _i, _vp, C.POINTER(C.c_double), _vp])

EXPORTED = ["lsas_status_str", "lsas_check_config", "lsas_frame_bytes",
            "lsas_plan_create", "lsas_plan_set", "lsas_plan_set_pilot",
            "lsas_fft", "lsas_estimate", "lsas_demodulate", "lsas_run_frame",
            "lsas_run_frame_host", "lsas_mrc_partial", "lsas_mrc_combine",
            "lsas_run_frame_split_static", "lsas_fft_tc", "lsas_fft_tc_ex", "lsas_receive_y",
            "lsas_plan_set_pn", "lsas_pn_sync", "lsas_pn_extract", "lsas_fftshift",
            "lsas_server_create", "lsas_server_register", "lsas_server_submit",
            "lsas_server_wait", "lsas_server_stats", "lsas_server_destroy",
            "lsas_server_submit_many", "lsas_server_wait_many",
            "lsas_server_register_refined", "lsas_server_set_admission",
            "lsas_server_frame_bytes",
            "lsas_dn_work_size", "lsas_dn_apply", "lsas_dn_grad", "lsas_dn_adam",
            "lsas_dn_to_bf16", "lsas_dn_apply_tc", "lsas_plan_set_fault",
            "lsas_plan_set_batch_split", "lsas_plan_batch_split_shards",
            "lsas_run_frame_refined", "lsas_dn_grad_tc",
            "lsas_plan_set_profile", "lsas_plan_profile",
            "lsas_plan_sync", "lsas_plan_info", "lsas_plan_device_bytes",
            "lsas_plan_destroy", "lsas_fma_peak_run"]


class LsasError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {lsas_status_str(code).decode()}")


def check(code: int, what: str = "lsas") -> None:
    if code != LSAS_OK:
        raise LsasError(code, what)


def frame_bytes(M, N, cp, n_sym, qam_order, fmt="sc16"):
    out = (C.c_size_t * 4)()
    check(lsas_frame_bytes(M, N, cp, n_sym, qam_order, _fmt(fmt), out), "lsas_frame_bytes")
    return tuple(int(v) for v in out)


def _fmt(fmt) -> int:
    if fmt in ("sc16", LSAS_IN_SC16):
        return LSAS_IN_SC16
    if fmt in ("fc32", LSAS_IN_FC32):
        return LSAS_IN_FC32
    raise ValueError(f"unknown input format {fmt!r}")


def _ptr(t) -> Optional[int]:
    return None if t is None else t.data_ptr()


def _stream(stream) -> Optional[int]:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream or None


def gather_partials(P, E, group=None):
    """Antenna split across processes (one shard of antennas per rank): every
    rank passes its shard's partial sums P [F][D][N] complex64 and E [F][N]
    float32 from Plan.mrc_partial and gets back all ranks' partials stacked in
    rank order, [world][F][D][N] and [world][F][N], for Plan.mrc_combine, which
    adds them in that fixed order.  Moves D*N complex + N real per frame and
    rank, against M*S*(N+CP) input samples."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    Pr = torch.view_as_real(P.contiguous())
    outP = [torch.empty_like(Pr) for _ in range(world)]
    outE = [torch.empty_like(E) for _ in range(world)]
    dist.all_gather(outP, Pr, group=group)
    dist.all_gather(outE, E.contiguous(), group=group)
    return torch.view_as_complex(torch.stack(outP)), torch.stack(outE)


class Plan:
    """A receiver configuration bound to the current CUDA device.

    Tensors: input ``[F][M][S*(N+CP)][2]`` int16 (sc16) or float32 (fc32);
    H and eq complex64; bits uint8 ``[F][D*N*q/8]``.
    """

    def __init__(self, M: int, N: int, cp: int, n_sym: int, pilot_idx: int = 0,
                 qam_order: int = 4, fmt: str = "sc16", max_frames: int = 1024,
                 pilot=None):
        self.M, self.N, self.cp, self.S = M, N, cp, n_sym
        self.pilot_idx, self.Q, self.fmt = pilot_idx, qam_order, fmt
        self.D = n_sym - 1
        self.q = int(round(np.log2(qam_order)))
        h = _vp()
        check(lsas_plan_create(M, N, cp, n_sym, pilot_idx, qam_order, C.byref(h)),
              "lsas_plan_create")
        self._h = h
        check(lsas_plan_set(self._h, _fmt(fmt), max_frames), "lsas_plan_set")
        self.max_frames = max_frames
        if pilot is not None:
            self.set_pilot(pilot)

    # ---- configuration
    def set_pilot(self, pilot) -> None:
        x = np.asarray(pilot, dtype=np.complex128)
        iq = np.ascontiguousarray(np.stack([x.real, x.imag], -1).astype(np.float32))
        check(lsas_plan_set_pilot(self._h, iq.ctypes.data_as(C.POINTER(_f))),
              "lsas_plan_set_pilot")

    def info(self) -> dict:
        out = (_i * 8)()
        check(lsas_plan_info(self._h, out), "lsas_plan_info")
        keys = ["antennas_per_step", "threads", "smem_bytes", "groups", "slots",
                "tma", "fmt", "max_frames"]
        return dict(zip(keys, list(out)))

    def set_batch_split(self, enable) -> None:
        """lsas_plan_set_batch_split: whether lsas_run_frame may split the
        frames after a batch's last whole wave into antenna shards (True or
        1: shard count per batch size; 2: one shard count for every batch;
        False or 0: never)."""
        mode = int(enable) if not isinstance(enable, bool) else (1 if enable else 0)
        check(lsas_plan_set_batch_split(self._h, mode), "lsas_plan_set_batch_split")

    def batch_split_shards(self, n_frames: int) -> int:
        """lsas_plan_batch_split_shards: the antenna shards lsas_run_frame
        would use for the frames after the last whole wave (1: none)."""
        out = _i(0)
        check(lsas_plan_batch_split_shards(self._h, int(n_frames), C.byref(out)),
              "lsas_plan_batch_split_shards")
        return int(out.value)

    def device_bytes(self) -> int:
        """lsas_plan_device_bytes: device memory the plan allocated at
        creation (tables and the split-tail scratch)."""
        out = C.c_size_t(0)
        check(lsas_plan_device_bytes(self._h, C.byref(out)), "lsas_plan_device_bytes")
        return int(out.value)

    def run_frame_launches(self, n_frames: int) -> int:
        """Kernel launches lsas_run_frame makes for an n_frames batch: one,
        or, when the frames after the last whole wave run split, the
        whole-wave launch (if there is a whole wave), the shard launch and
        the combine pass."""
        if self.batch_split_shards(n_frames) == 1:
            return 1
        import torch
        sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
        return (1 if n_frames >= sms else 0) + 2

    @property
    def handle(self):
        return self._h

    # ---- buffers
    def _frames(self, x) -> int:
        if not x.is_contiguous():
            raise ValueError("input must be contiguous")
        want = np.int16 if self.fmt == "sc16" else np.float32
        import torch
        tdt = torch.int16 if want == np.int16 else torch.float32
        if x.dtype != tdt:
            raise TypeError(f"input dtype must be {tdt} for {self.fmt}")
        per = self.M * self.S * (self.N + self.cp) * 2
        if x.numel() % per:
            raise ValueError("input size is not a whole number of frames")
        return x.numel() // per

    def empty_H(self, F, device="cuda"):
        import torch
        return torch.empty((F, self.M, self.N), dtype=torch.complex64, device=device)

    def empty_bits(self, F, device="cuda"):
        import torch
        return torch.empty((F, self.D * self.N * self.q // 8), dtype=torch.uint8, device=device)

    def empty_eq(self, F, device="cuda"):
        import torch
        return torch.empty((F, self.D, self.N), dtype=torch.complex64, device=device)

    # ---- operations
    def fft(self, x, Y=None, stream=None):
        import torch
        F = self._frames(x)
        if Y is None:
            Y = torch.empty((F, self.M, self.S, self.N), dtype=torch.complex64, device=x.device)
        check(lsas_fft(self._h, _ptr(x), F, _ptr(Y), _stream(stream)), "lsas_fft")
        return Y

    def fft_tc(self, x, terms=3, Y=None, stream=None, operand="fp16"):
        """The FFT on the tensor cores (fp16 or bf16 operands; terms=3 splits
        them into hi + lo parts), Y [F][M][S][N] complex64."""
        import torch
        F = self._frames(x)
        if Y is None:
            Y = torch.empty((F, self.M, self.S, self.N), dtype=torch.complex64, device=x.device)
        op = {"fp16": LSAS_TC_FP16, "bf16": LSAS_TC_BF16}[operand]
        check(lsas_fft_tc_ex(self._h, _ptr(x), F, op, terms, _ptr(Y), _stream(stream)),
              "lsas_fft_tc_ex")
        return Y

    def receive_y(self, Y, H=None, bits=None, eq=None, want_eq=False, stream=None):
        """LS, MRC and demap from transformed symbols Y [F][M][S][N]."""
        F = int(Y.shape[0])
        if not Y.is_contiguous() or tuple(Y.shape[1:]) != (self.M, self.S, self.N):
            raise ValueError("Y must be a contiguous [F][M][S][N] complex64 tensor")
        H = self.empty_H(F, Y.device) if H is None else H
        bits = self.empty_bits(F, Y.device) if bits is None else bits
        if eq is None and want_eq:
            eq = self.empty_eq(F, Y.device)
        check(lsas_receive_y(self._h, _ptr(Y), F, _ptr(H), _ptr(bits), _ptr(eq), _stream(stream)),
              "lsas_receive_y")
        return H, bits, eq

    # ---- packet detection and output order
    def set_pn(self, pn) -> None:
        chips = np.ascontiguousarray(np.asarray(pn, dtype=np.float32))
        check(lsas_plan_set_pn(self._h, chips.ctypes.data_as(C.POINTER(_f)), int(chips.size)),
              "lsas_plan_set_pn")
        self.pn_len = int(chips.size)

    def pn_sync(self, cap, window, offsets=None, peaks=None, stream=None):
        """Preamble start per frame of captures cap [F][M][Lc][2]: (offsets, peaks)."""
        import torch
        if not cap.is_contiguous() or cap.dim() != 4 or cap.shape[1] != self.M:
            raise ValueError("captures must be a contiguous [F][M][Lc][2] tensor")
        F, Lc = int(cap.shape[0]), int(cap.shape[2])
        offsets = torch.empty(F, dtype=torch.int32, device=cap.device) if offsets is None else offsets
        peaks = torch.empty(F, dtype=torch.float32, device=cap.device) if peaks is None else peaks
        check(lsas_pn_sync(self._h, _ptr(cap), F, Lc, window, _ptr(offsets), _ptr(peaks),
                           _stream(stream)), "lsas_pn_sync")
        return offsets, peaks

    def pn_extract(self, cap, offsets, backoff=0, frames=None, stream=None):
        """Frames [F][M][S(N+CP)][2] cut out of the captures after the preamble."""
        import torch
        F, Lc = int(cap.shape[0]), int(cap.shape[2])
        if frames is None:
            frames = torch.empty((F, self.M, self.S * (self.N + self.cp), 2), dtype=cap.dtype,
                                 device=cap.device)
        check(lsas_pn_extract(self._h, _ptr(cap), F, Lc, _ptr(offsets), backoff, _ptr(frames),
                              _stream(stream)), "lsas_pn_extract")
        return frames

    def fftshift(self, what, buf, stream=None):
        """In-place fftshift of an output buffer (what = LSAS_SHIFT_*)."""
        check(lsas_fftshift(self._h, what, _ptr(buf), int(buf.shape[0]), _stream(stream)),
              "lsas_fftshift")
        return buf

    def estimate(self, x, H=None, stream=None):
        F = self._frames(x)
        H = self.empty_H(F, x.device) if H is None else H
        check(lsas_estimate(self._h, _ptr(x), F, _ptr(H), _stream(stream)), "lsas_estimate")
        return H

    def demodulate(self, x, H, bits=None, eq=None, want_eq=False, stream=None):
        F = self._frames(x)
        bits = self.empty_bits(F, x.device) if bits is None else bits
        if eq is None and want_eq:
            eq = self.empty_eq(F, x.device)
        check(lsas_demodulate(self._h, _ptr(x), _ptr(H), F, _ptr(bits), _ptr(eq),
                              _stream(stream)), "lsas_demodulate")
        return bits, eq

    def run_frame_refined(self, x, params_bf16, work, status, H=None, bits=None, eq=None,
                          want_eq=False, stream=None):
        """lsas_run_frame_refined: LS fused with the tensor-core refinement,
        then MRC and demap with the refined channel (N = 1024, sc16)."""
        F = self._frames(x)
        H = self.empty_H(F, x.device) if H is None else H
        bits = self.empty_bits(F, x.device) if bits is None else bits
        if eq is None and want_eq:
            eq = self.empty_eq(F, x.device)
        check(lsas_run_frame_refined(self._h, _ptr(x), F, _ptr(params_bf16), _ptr(work), _ptr(H),
                                     _ptr(bits), _ptr(eq), _ptr(status), _stream(stream)),
              "lsas_run_frame_refined")
        return H, bits, eq

    def run_frame(self, x, H=None, bits=None, eq=None, want_eq=False, stream=None):
        F = self._frames(x)
        H = self.empty_H(F, x.device) if H is None else H
        bits = self.empty_bits(F, x.device) if bits is None else bits
        if eq is None and want_eq:
            eq = self.empty_eq(F, x.device)
        check(lsas_run_frame(self._h, _ptr(x), F, _ptr(H), _ptr(bits), _ptr(eq),
                             _stream(stream)), "lsas_run_frame")
        return H, bits, eq

    def host_input_bytes_per_frame(self) -> int:
        """Input bytes per frame that lsas_run_frame_host moves over the host
        link: the samples after each cyclic prefix once a row of N samples
        spans at least 1 KB, else whole rows."""
        bps = 4 if self.fmt == "sc16" else 8
        strip = self.cp > 0 and self.N * bps >= 1024
        return self.M * self.S * (self.N if strip else self.N + self.cp) * bps

    def run_frame_host(self, x, H, bits, eq=None, stream=None):
        """Host (pinned) tensors in and out; copies happen inside the call."""
        F = self._frames(x)
        check(lsas_run_frame_host(self._h, _ptr(x), F, _ptr(H), _ptr(bits), _ptr(eq),
                                  _stream(stream)), "lsas_run_frame_host")
        return H, bits, eq

    def run_frame_split(self, x, n_shards, H=None, bits=None, eq=None, want_eq=False, stream=None):
        """lsas_run_frame_split_static: the antenna-split receiver with its
        partial sums in the library's fixed scratch.  With equal shards (M a
        multiple of n_shards, N <= 1024) one launch runs every shard of a
        frame side by side, which cuts the latency of small batches."""
        F = self._frames(x)
        H = self.empty_H(F, x.device) if H is None else H
        bits = self.empty_bits(F, x.device) if bits is None else bits
        if eq is None and want_eq:
            eq = self.empty_eq(F, x.device)
        check(lsas_run_frame_split_static(self._h, _ptr(x), F, int(n_shards), _ptr(H), _ptr(bits),
                                          _ptr(eq), _stream(stream)), "lsas_run_frame_split_static")
        return H, bits, eq

    # ---- antenna split (shard partial sums, then a fixed-order combine)
    def empty_partials(self, F, shards=1, device="cuda"):
        """Zeroed P [shards][F][D][N] complex64 and E [shards][F][N] float32."""
        import torch
        return (torch.zeros((shards, F, self.D, self.N), dtype=torch.complex64, device=device),
                torch.zeros((shards, F, self.N), dtype=torch.float32, device=device))

    def mrc_partial(self, x, m_begin, m_count, H, P, E, stream=None):
        """Antennas [m_begin, m_begin + m_count): writes their rows of H and the
        shard's partial sums P [F][D][N], E [F][N]."""
        F = self._frames(x)
        check(lsas_mrc_partial(self._h, _ptr(x), F, m_begin, m_count, _ptr(H), _ptr(P),
                               _ptr(E), _stream(stream)), "lsas_mrc_partial")
        return H, P, E

    def mrc_combine(self, P, E, bits=None, eq=None, want_eq=False, stream=None):
        """Adds the shards of P [G][F][D][N] and E [G][F][N] in order, then
        slices and packs; returns (bits, eq)."""
        G, F = int(P.shape[0]), int(P.shape[1])
        if not (P.is_contiguous() and E.is_contiguous()):
            raise ValueError("partials must be contiguous")
        if tuple(E.shape) != (G, F, self.N) or tuple(P.shape[2:]) != (self.D, self.N):
            raise ValueError("partials have the wrong shape")
        bits = self.empty_bits(F, P.device) if bits is None else bits
        if eq is None and want_eq:
            eq = self.empty_eq(F, P.device)
        check(lsas_mrc_combine(self._h, _ptr(P), _ptr(E), G, F, _ptr(bits), _ptr(eq),
                               _stream(stream)), "lsas_mrc_combine")
        return bits, eq

    def set_profile(self, on: bool = True) -> None:
        """Time every library call on this plan (CUDA events on its stream)."""
        check(lsas_plan_set_profile(self._h, 1 if on else 0), "lsas_plan_set_profile")

    def profile(self) -> dict:
        """Per-function call counts and device milliseconds since the last
        read: {"lsas_run_frame": {"calls": n, "ms": t}, ...}; clears them."""
        import json
        need = C.c_size_t()
        check(lsas_plan_profile(self._h, None, 0, C.byref(need)), "lsas_plan_profile")
        buf = C.create_string_buffer(need.value + 256)
        check(lsas_plan_profile(self._h, buf, len(buf), C.byref(need)), "lsas_plan_profile")
        return json.loads(buf.value.decode())

    def sync(self, stream=None) -> None:
        """Synchronise and raise if a device-side condition was latched."""
        check(lsas_plan_sync(self._h, _stream(stream)), "device status")

    def sync_status(self, stream=None) -> int:
        return lsas_plan_sync(self._h, _stream(stream))

    def close(self) -> None:
        if getattr(self, "_h", None):
            lsas_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Serving loop: frames of registered configurations in host memory,
    batched per configuration and run on the fused receiver.  Host tensors
    passed to submit() are kept alive here until their wait() returns."""

    def __init__(self, mem_budget: int, max_batch: int = 32, max_wait_us: float = 200.0):
        h = _vp()
        check(lsas_server_create(int(mem_budget), max_batch, float(max_wait_us), C.byref(h)),
              "lsas_server_create")
        self._h = h
        self._live = {}
        self._params = []
        self.configs = {}

    def register(self, M, N, cp, n_sym, pilot_idx=0, qam_order=4, fmt="sc16", pilot=None,
                 refine_params_bf16=None) -> int:
        """Register a configuration; with ``refine_params_bf16`` (a device
        tensor of LSAS_DN_PARAMS bf16 values, kept alive here) its frames run
        the learned form (LS -> tensor-core refinement -> MRC)."""
        ptr = None
        if pilot is not None:
            x = np.asarray(pilot, dtype=np.complex128)
            iq = np.ascontiguousarray(np.stack([x.real, x.imag], -1).astype(np.float32))
            ptr = iq.ctypes.data_as(C.POINTER(_f))
        cid = _i()
        if refine_params_bf16 is None:
            check(lsas_server_register(self._h, M, N, cp, n_sym, pilot_idx, qam_order, _fmt(fmt),
                                       ptr, C.byref(cid)), "lsas_server_register")
        else:
            check(lsas_server_register_refined(self._h, M, N, cp, n_sym, pilot_idx, qam_order,
                                               _fmt(fmt), ptr, _ptr(refine_params_bf16),
                                               C.byref(cid)), "lsas_server_register_refined")
            self._params.append(refine_params_bf16)
        q = int(round(np.log2(qam_order)))
        self.configs[cid.value] = dict(M=M, N=N, cp=cp, S=n_sym, D=n_sym - 1, q=q,
                                       refined=refine_params_bf16 is not None)
        return cid.value

    def set_admission(self, frame_budget_bytes: int = 0, wait_ms: float = 0.0) -> None:
        check(lsas_server_set_admission(self._h, int(frame_budget_bytes), float(wait_ms)),
              "lsas_server_set_admission")

    def frame_bytes(self) -> dict:
        out = (C.c_uint64 * 2)()
        check(lsas_server_frame_bytes(self._h, out), "lsas_server_frame_bytes")
        return dict(charged=int(out[0]), budget=int(out[1]))

    def submit(self, cid, x, H, bits, eq=None) -> int:
        t = C.c_uint64()
        check(lsas_server_submit(self._h, cid, _ptr(x), _ptr(H), _ptr(bits), _ptr(eq), C.byref(t)),
              "lsas_server_submit")
        self._live[t.value] = (x, H, bits, eq)
        return t.value

    def wait(self, ticket, timeout_ms=30000.0) -> float:
        lat = C.c_double()
        code = lsas_server_wait(self._h, ticket, float(timeout_ms), C.byref(lat))
        if code != LSAS_ERR_TIMEOUT:
            self._live.pop(ticket, None)
        check(code, "lsas_server_wait")
        return lat.value

    def submit_many(self, frames) -> list:
        """frames: sequence of (config_id, x, H, bits[, eq]); one call queues
        them all (or none) and returns their tickets in order."""
        n = len(frames)
        if n == 0:
            return []
        cids = (_i * n)(*[int(f[0]) for f in frames])
        xs = (_vp * n)(*[_ptr(f[1]) for f in frames])
        Hs = (_vp * n)(*[_ptr(f[2]) for f in frames])
        bs = (_vp * n)(*[_ptr(f[3]) for f in frames])
        eqs = [f[4] if len(f) > 4 else None for f in frames]
        es = (_vp * n)(*[_ptr(e) for e in eqs]) if any(e is not None for e in eqs) else None
        t = (C.c_uint64 * n)()
        check(lsas_server_submit_many(self._h, n, cids, xs, Hs, bs, es, t), "lsas_server_submit_many")
        for i, f in enumerate(frames):
            self._live[t[i]] = (f[1], f[2], f[3], eqs[i])
        return list(t)

    def wait_many(self, tickets, timeout_ms=30000.0) -> list:
        """Wait for all tickets; their submit-to-results latencies (us)."""
        n = len(tickets)
        if n == 0:
            return []
        t = (C.c_uint64 * n)(*tickets)
        lat = (C.c_double * n)()
        code = lsas_server_wait_many(self._h, n, t, float(timeout_ms), lat, None)
        if code != LSAS_ERR_TIMEOUT and code != LSAS_ERR_INVALID_ARG:
            for k in tickets:
                self._live.pop(k, None)
        check(code, "lsas_server_wait_many")
        return list(lat)

    def stats(self) -> dict:
        out = (C.c_uint64 * 4)()
        check(lsas_server_stats(self._h, out), "lsas_server_stats")
        return dict(launches=int(out[0]), frames=int(out[1]), admitted_bytes=int(out[2]),
                    configs=int(out[3]))

    def set_batch_split(self, enable) -> None:
        """lsas_plan_set_batch_split: whether lsas_run_frame may split the
        frames after a batch's last whole wave into antenna shards (True or
        1: shard count per batch size; 2: one shard count for every batch;
        False or 0: never)."""
        mode = int(enable) if not isinstance(enable, bool) else (1 if enable else 0)
        check(lsas_plan_set_batch_split(self._h, mode), "lsas_plan_set_batch_split")

    def batch_split_shards(self, n_frames: int) -> int:
        """lsas_plan_batch_split_shards: the antenna shards lsas_run_frame
        would use for the frames after the last whole wave (1: none)."""
        out = _i(0)
        check(lsas_plan_batch_split_shards(self._h, int(n_frames), C.byref(out)),
              "lsas_plan_batch_split_shards")
        return int(out.value)

    @property
    def handle(self):
        return self._h

    def close(self) -> int:
        code = LSAS_OK
        if getattr(self, "_h", None):
            code = lsas_server_destroy(self._h)
            self._h = None
            self._live.clear()
        return code

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
