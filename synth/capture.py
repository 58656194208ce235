"""Seeded captures with a PN preamble (transmitter + channel + front-end).

The paper's transmitter (Sec. II-B) sends a maximum-length PN sequence for
packet detection, then the OFDM frame (channel-estimation symbol first, then
the data symbols).  A capture here is what one antenna records around one
such transmission: ``delay`` samples before the preamble starts, the 255-chip
preamble, the frame, and silence after it, through the same block-fading
multipath channel and AWGN as ``synth.frames``.  The receiver must find the
preamble (PN correlation) to know where the frame begins.

* PN sequence: the m-sequence of the primitive polynomial
  x^8 + x^4 + x^3 + x^2 + 1, a[n + 8] = a[n + 4] ^ a[n + 3] ^ a[n + 2] ^ a[n],
  a[0..7] = 1, 0, ..., 0, mapped 0 -> +1, 1 -> -1 (BPSK chips of unit power).
* Every draw of capture ``f`` comes from ``default_rng([seed, f, 0x504e])``;
  the delay is uniform on [0, max_delay).
* Capture length ``max_delay + 255 + S (N + CP)``; the frame starts at sample
  ``delay + 255``.
* sc16 scaling as in ``synth.frames`` (RMS 2048 over the samples that carry
  signal, the same gain applied to the whole capture).
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .frames import FrameConfig, pdp, pilot_sequence, qam_map

PN_LEN = 255


def pn_sequence() -> np.ndarray:
    """The 255 BPSK chips (+1 / -1) of the degree-8 m-sequence."""
    a = np.zeros(PN_LEN + 8, dtype=np.int64)
    a[0] = 1
    for n in range(PN_LEN):
        a[n + 8] = a[n + 4] ^ a[n + 3] ^ a[n + 2] ^ a[n]
    return 1.0 - 2.0 * a[:PN_LEN].astype(np.float64)


@dataclass
class CaptureBatch:
    cfg: FrameConfig
    ids: np.ndarray
    captures: np.ndarray      # [F][M][Lc][2] int16 or float32
    delay: np.ndarray         # [F] preamble start (samples)
    frame_start: np.ndarray   # [F] = delay + 255
    pilot: np.ndarray
    pn: np.ndarray
    bits: np.ndarray          # [F][D][N][q]
    X: np.ndarray             # [F][S][N]
    taps: np.ndarray          # [F][M][L] channel taps
    max_delay: int


def capture_length(cfg: FrameConfig, max_delay: int) -> int:
    return max_delay + PN_LEN + cfg.S * (cfg.N + cfg.cp)


def _one_capture(cfg: FrameConfig, f: int, pilot: np.ndarray, pn: np.ndarray, max_delay: int):
    rng = np.random.default_rng([cfg.seed, int(f), 0x504E])
    N, cp, S, M, D, q = cfg.N, cfg.cp, cfg.S, cfg.M, cfg.D, cfg.q
    bits = rng.integers(0, 2, size=(D, N, q), dtype=np.uint8)
    X = np.empty((S, N), dtype=np.complex128)
    data_syms = [s for s in range(S) if s != cfg.pilot_idx]
    X[cfg.pilot_idx] = pilot
    X[data_syms] = qam_map(bits, cfg.Q)
    x = np.fft.ifft(X, axis=-1) * np.sqrt(N)
    x = np.concatenate([x[:, N - cp:], x], axis=-1).reshape(-1)
    delay = int(rng.integers(0, max_delay))
    Lc = capture_length(cfg, max_delay)
    s = np.zeros(Lc, dtype=np.complex128)
    s[delay:delay + PN_LEN] = pn
    s[delay + PN_LEN:delay + PN_LEN + x.shape[0]] = x
    p = pdp(cfg.taps, cfg.decay_db)
    h = (rng.standard_normal((M, cfg.taps)) +
         1j * rng.standard_normal((M, cfg.taps))) * np.sqrt(p / 2.0)
    y = np.zeros((M, Lc), dtype=np.complex128)
    for l in range(cfg.taps):
        y[:, l:] += h[:, l:l + 1] * s[None, :Lc - l]
    if cfg.snr_db is not None:
        snr = float(rng.uniform(*cfg.snr_db)) if isinstance(cfg.snr_db, tuple) else float(cfg.snr_db)
        s2 = 10.0 ** (-snr / 10.0)
        w = rng.standard_normal((M, Lc, 2)) * np.sqrt(s2 / 2.0)
        y = y + (w[..., 0] + 1j * w[..., 1])
    if cfg.fmt == "sc16":
        active = y[:, delay:delay + PN_LEN + x.shape[0]]
        g = 2048.0 / np.sqrt(np.mean(np.abs(active) ** 2))
        iq = np.stack([np.rint(g * y.real), np.rint(g * y.imag)], axis=-1)
        out = np.clip(iq, -32767, 32767).astype(np.int16)
    else:
        out = np.stack([y.real, y.imag], axis=-1).astype(np.float32)
    return out, delay, bits, X, h


def generate_capture(cfg: FrameConfig, frame_ids=None, max_delay: int = 512) -> CaptureBatch:
    if frame_ids is None:
        frame_ids = range(cfg.F)
    ids = np.asarray(list(frame_ids), dtype=np.int64)
    pil = pilot_sequence(cfg)
    pn = pn_sequence()
    F = ids.shape[0]
    dt = np.int16 if cfg.fmt == "sc16" else np.float32
    Lc = capture_length(cfg, max_delay)
    caps = np.empty((F, cfg.M, Lc, 2), dtype=dt)
    delay = np.empty(F, dtype=np.int64)
    bits = np.empty((F, cfg.D, cfg.N, cfg.q), dtype=np.uint8)
    X = np.empty((F, cfg.S, cfg.N), dtype=np.complex128)
    taps = np.empty((F, cfg.M, cfg.taps), dtype=np.complex128)
    for i, f in enumerate(ids):
        caps[i], delay[i], bits[i], X[i], taps[i] = _one_capture(cfg, int(f), pil, pn, max_delay)
    return CaptureBatch(cfg, ids, caps, delay, delay + PN_LEN, pil, pn, bits, X, taps, max_delay)
