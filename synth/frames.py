"""Seeded OFDM uplink frame generator (transmitter + channel + front-end).

Every random draw of frame ``f`` comes from its own stream
``numpy.random.default_rng([seed, f])``, so any subset of frames can be
regenerated bit-identically in any order.  The pilot comes from the stream
``[seed, 0x7fffffff, 1]`` and is the same for every frame, as the receiver must
know it (Sec. II-B: the first symbol is the channel-estimation symbol).

Conventions (they fix what the receiver must recover):

* Gray square QAM, unit average energy.  Per axis, ``L = sqrt(Q)`` levels at
  ``(2 i - (L - 1)) * A`` with ``A = 1 / sqrt(2 (Q - 1) / 3)``; level ``i``
  carries the Gray word ``i ^ (i >> 1)`` written MSB-first, I-axis bits first.
  BPSK (Q = 2) uses the I axis only, levels -1 and +1.
* Unitary OFDM modulation: ``x[n] = N**-0.5 * sum_k X[k] exp(+2j pi k n / N)``.
* Channel per antenna: ``taps`` taps at one-sample spacing, tap ``l`` drawn
  CN(0, p_l) with an exponential power-delay profile of ``decay_db`` per tap,
  normalised so that the expected total power is 1.  Block fading over a frame;
  the frame stream is convolved with zero history before the frame.
* AWGN CN(0, sigma^2) with ``sigma^2 = 10**(-snr_db / 10)`` per time-domain
  sample, relative to the expected received power 1.
* sc16: per frame, gain ``g = 2048 / rms(y)`` over all antennas and samples,
  ``I = clip(rint(g Re y), -32767, 32767)`` (round half to even), same for Q.
"""

from __future__ import annotations

import dataclasses
from dataclasses import dataclass, field
from typing import Optional, Sequence, Tuple, Union

import numpy as np

BASE_SEED = 0x190107499


@dataclass(frozen=True)
class FrameConfig:
    """Shape and channel statistics of a batch of received frames."""
    M: int                      # receive antennas
    N: int                      # FFT length = subcarriers
    cp: int                     # cyclic prefix length (samples)
    S: int                      # OFDM symbols per frame (1 pilot + S-1 data)
    Q: int                      # QAM order of the data symbols
    pilot_idx: int = 0          # index of the channel-estimation symbol
    taps: int = 4               # channel taps per antenna
    decay_db: float = 3.0       # exponential power-delay profile, dB per tap
    snr_db: Union[float, Tuple[float, float], None] = 20.0  # None = noiseless
    fmt: str = "fc32"           # "fc32" or "sc16"
    F: int = 16                 # frames in the full workload
    seed: int = BASE_SEED
    name: str = "custom"

    @property
    def D(self) -> int:
        return self.S - 1

    @property
    def q(self) -> int:
        return int(round(np.log2(self.Q)))

    @property
    def T(self) -> int:
        """Time-domain samples per antenna per frame."""
        return self.S * (self.N + self.cp)

    def replace(self, **kw) -> "FrameConfig":
        return dataclasses.replace(self, **kw)


def _named(name, **kw):
    return FrameConfig(name=name, **kw)


# The workloads: the paper's antenna-count / FFT-length grid (Table I, Sec. III)
# at its two FFT lengths, and the scaled-up shapes the library is measured on.
CONFIGS = {
    # 8 antennas, N=64, CP=16, 1 pilot + 14 QPSK, 4-tap 3 dB/tap, 20 dB, fc32
    "tiny": _named("tiny", M=8, N=64, cp=16, S=15, Q=4, taps=4, decay_db=3.0,
                   snr_db=20.0, fmt="fc32", F=16, seed=BASE_SEED + 1),
    # 64 antennas, N=1024, CP=128, 1 pilot + 13 16-QAM, 8-tap 2 dB/tap,
    # SNR uniform 10..30 dB per frame, sc16, 1000 frames
    "scale": _named("scale", M=64, N=1024, cp=128, S=14, Q=16, taps=8,
                    decay_db=2.0, snr_db=(10.0, 30.0), fmt="sc16", F=1000,
                    seed=BASE_SEED + 2),
    # 128 antennas, N=2048, CP=256, 1 pilot + 13 64-QAM, 16-tap 1 dB/tap,
    # 30 dB, sc16, 500 frames
    "precision": _named("precision", M=128, N=2048, cp=256, S=14, Q=64,
                        taps=16, decay_db=1.0, snr_db=30.0, fmt="sc16", F=500,
                        seed=BASE_SEED + 3),
}


def sweep_config(M: int, N: int, F: int = 1000) -> FrameConfig:
    """One point of the antenna x FFT-length sweep (CP = N/8, as "scale")."""
    base = CONFIGS["scale"]
    return base.replace(M=M, N=N, cp=N // 8, F=F, name=f"sweep_M{M}_N{N}")


def paper_config(M: int, N: int, F: int = 8) -> FrameConfig:
    """The paper's own shapes: N=64 with CP 16, N=1024 with CP 72 (Table I)."""
    cp = {64: 16, 1024: 72}[N]
    return CONFIGS["scale"].replace(M=M, N=N, cp=cp, Q=16, F=F,
                                    name=f"paper_M{M}_N{N}")


def config_by_name(name: str) -> FrameConfig:
    if name in CONFIGS:
        return CONFIGS[name]
    if name.startswith("sweep_M"):
        m, n = name[len("sweep_M"):].split("_N")
        return sweep_config(int(m), int(n))
    raise KeyError(name)


# --------------------------------------------------------------------------
# Transmitter
# --------------------------------------------------------------------------

def gray_levels(Q: int) -> Tuple[int, float]:
    """Levels per axis and the amplitude unit A of unit-energy square QAM."""
    if Q == 2:
        return 2, 1.0
    L = int(round(np.sqrt(Q)))
    if L * L != Q or L < 2 or (L & (L - 1)):
        raise ValueError(f"unsupported QAM order {Q}")
    return L, 1.0 / np.sqrt(2.0 * (Q - 1) / 3.0)


def _gray_to_level(bits: np.ndarray) -> np.ndarray:
    """bits [..., w] MSB-first Gray word -> level index (inverse Gray code)."""
    w = bits.shape[-1]
    g = np.zeros(bits.shape[:-1], dtype=np.int64)
    for j in range(w):
        g = (g << 1) | bits[..., j].astype(np.int64)
    lvl = g.copy()
    shift = g >> 1
    while np.any(shift):
        lvl ^= shift
        shift >>= 1
    return lvl


def qam_map(bits: np.ndarray, Q: int) -> np.ndarray:
    """Map bits [..., q] to unit-energy Gray QAM symbols (complex128)."""
    L, A = gray_levels(Q)
    if Q == 2:
        lvl = bits[..., 0].astype(np.int64)
        return ((2 * lvl - 1) * A).astype(np.complex128)
    w = int(np.log2(L))
    li = _gray_to_level(bits[..., :w])
    lq = _gray_to_level(bits[..., w:2 * w])
    return ((2 * li - (L - 1)) * A + 1j * ((2 * lq - (L - 1)) * A))


def pilot_sequence(cfg: FrameConfig) -> np.ndarray:
    """The known +-1 BPSK pilot on all N subcarriers (complex128 [N])."""
    rng = np.random.default_rng([cfg.seed, 0x7FFFFFFF, 1])
    return (2.0 * rng.integers(0, 2, size=cfg.N) - 1.0).astype(np.complex128)


def pdp(taps: int, decay_db: float) -> np.ndarray:
    p = 10.0 ** (-decay_db * np.arange(taps) / 10.0)
    return p / p.sum()


@dataclass
class FrameBatch:
    cfg: FrameConfig
    frame_ids: np.ndarray       # [F] frame indices into the seeded stream
    frames: np.ndarray          # [F][M][T][2] int16 (sc16) or float32 (fc32)
    pilot: np.ndarray           # [N] complex128
    bits: np.ndarray            # [F][D][N][q] uint8, transmitted data bits
    X: np.ndarray               # [F][S][N] complex128 transmitted subcarriers
    taps: np.ndarray            # [F][M][L] complex128 channel taps
    gain: np.ndarray            # [F] front-end gain g (1 for fc32)
    snr_db: np.ndarray          # [F]
    sigma2: np.ndarray          # [F]
    clips: np.ndarray           # [F] clipped int16 components (sc16)

    @property
    def F(self) -> int:
        return self.frames.shape[0]

    def as_complex(self) -> np.ndarray:
        """Received samples as complex128 [F][M][T] (exact int16 -> double)."""
        f = self.frames.astype(np.float64)
        return f[..., 0] + 1j * f[..., 1]


def _one_frame(cfg: FrameConfig, f: int, pilot: np.ndarray,
               taps_override: Optional[np.ndarray]):
    rng = np.random.default_rng([cfg.seed, int(f)])
    N, cp, S, M, D = cfg.N, cfg.cp, cfg.S, cfg.M, cfg.D
    q = cfg.q
    bits = rng.integers(0, 2, size=(D, N, q), dtype=np.uint8)
    X = np.empty((S, N), dtype=np.complex128)
    data_syms = [s for s in range(S) if s != cfg.pilot_idx]
    X[cfg.pilot_idx] = pilot
    X[data_syms] = qam_map(bits, cfg.Q)
    # unitary OFDM modulation and cyclic prefix
    x = np.fft.ifft(X, axis=-1) * np.sqrt(N)
    x = np.concatenate([x[:, N - cp:], x], axis=-1).reshape(-1)   # [T]
    T = x.shape[0]
    # multipath Rayleigh channel per antenna
    p = pdp(cfg.taps, cfg.decay_db)
    h = (rng.standard_normal((M, cfg.taps)) +
         1j * rng.standard_normal((M, cfg.taps))) * np.sqrt(p / 2.0)
    if taps_override is not None:
        h = np.broadcast_to(np.asarray(taps_override, np.complex128),
                            (M, np.asarray(taps_override).shape[-1])).copy()
    L = h.shape[1]
    shifted = np.zeros((L, T), dtype=np.complex128)
    for l in range(L):
        shifted[l, l:] = x[:T - l]
    y = h @ shifted                                                  # [M][T]
    # AWGN
    if cfg.snr_db is None:
        snr, s2 = np.inf, 0.0
    else:
        if isinstance(cfg.snr_db, tuple):
            snr = float(rng.uniform(cfg.snr_db[0], cfg.snr_db[1]))
        else:
            snr = float(cfg.snr_db)
        s2 = 10.0 ** (-snr / 10.0)
        w = rng.standard_normal((M, T, 2)) * np.sqrt(s2 / 2.0)
        y = y + (w[..., 0] + 1j * w[..., 1])
    if cfg.fmt == "sc16":
        g = 2048.0 / np.sqrt(np.mean(np.abs(y) ** 2))
        iq = np.stack([np.rint(g * y.real), np.rint(g * y.imag)], axis=-1)
        clips = int(np.count_nonzero(np.abs(iq) > 32767))
        out = np.clip(iq, -32767, 32767).astype(np.int16)
    elif cfg.fmt == "fc32":
        g, clips = 1.0, 0
        out = np.stack([y.real, y.imag], axis=-1).astype(np.float32)
    else:
        raise ValueError(cfg.fmt)
    return out, bits, X, h, g, snr, s2, clips


def generate(cfg: FrameConfig, frame_ids: Optional[Sequence[int]] = None,
             taps: Optional[np.ndarray] = None,
             pilot: Optional[np.ndarray] = None) -> FrameBatch:
    """Generate the frames ``frame_ids`` (default ``range(cfg.F)``).

    ``taps`` overrides the random channel with fixed taps (same for every
    antenna unless given per antenna as [M][L]); ``pilot`` overrides the seeded
    +-1 pilot (any non-zero complex values).
    """
    if frame_ids is None:
        frame_ids = range(cfg.F)
    ids = np.asarray(list(frame_ids), dtype=np.int64)
    if taps is not None and np.asarray(taps).shape[-1] - 1 > cfg.cp:
        raise ValueError("channel longer than the cyclic prefix")
    pil = pilot_sequence(cfg) if pilot is None else np.asarray(pilot, np.complex128)
    dt = np.int16 if cfg.fmt == "sc16" else np.float32
    F = ids.shape[0]
    L = cfg.taps if taps is None else np.asarray(taps).shape[-1]
    frames = np.empty((F, cfg.M, cfg.T, 2), dtype=dt)
    bits = np.empty((F, cfg.D, cfg.N, cfg.q), dtype=np.uint8)
    X = np.empty((F, cfg.S, cfg.N), dtype=np.complex128)
    H = np.empty((F, cfg.M, L), dtype=np.complex128)
    gain = np.empty(F); snr = np.empty(F); s2 = np.empty(F)
    clips = np.empty(F, dtype=np.int64)
    for i, f in enumerate(ids):
        (frames[i], bits[i], X[i], H[i], gain[i], snr[i], s2[i],
         clips[i]) = _one_frame(cfg, int(f), pil, taps)
    return FrameBatch(cfg, ids, frames, pil, bits, X, H, gain, snr, s2, clips)
