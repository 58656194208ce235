"""FP64 CPU oracle of the uplink receiver: CP removal, FFT, LS, MRC, demap.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline legs of ``bench.py`` may import this module.  It is a plain, slow,
obviously correct restatement of the method in double precision; it shares no
code, table or constant with the CUDA library and never calls it.

What it computes, step by step, for one received frame of M antennas
(paper notation swapped: here M = antennas, N = FFT length / subcarriers):

1. CP removal (Sec. II-B): ``r[m, s, n] = y[m, s (N + CP) + CP + n]``.
2. FFT of every symbol of every antenna (Sec. II-B, Sec. II-C): the unitary DFT
   ``Y[m, s, k] = N**-0.5 sum_n r[m, s, n] exp(-2j pi k n / N)``, written out
   as its definition: a product with the N x N DFT matrix.
3. Least Squares estimate from the channel-estimation symbol (Sec. II-B,
   Sec. II-C): division by the known pilot, ``H = Y_p conj(X_p) / |X_p|^2``.
4. Maximal Ratio Combining over the antennas (Sec. II-C):
   ``z[d, k] = sum_m conj(H[m, k]) Y[m, s_d, k] / sum_m |H[m, k]|^2``; the
   conjugate and the channel-energy sum are formed once per frame and reused
   for every data symbol (Sec. III).  Zero energy gives ``z = 0`` and a flag.
5. Hard decision of each axis of ``z`` to the nearest Gray-QAM level and the
   level's Gray word (the demodulated output of Sec. II-B, in bits).

The antenna split of step 4 (the distributed receiver Sec. IV proposes):
each shard of antennas forms the two sums of step 4 over its own antennas;
the shards' partial sums are added and divided afterwards.

Upstream of step 1, packet detection (Sec. II-B): the received samples are
correlated with the known PN sequence; the power of the correlation, summed
over antennas, peaks where the preamble begins, and the frame follows it.
Downstream, the paper's fftshift (Sec. II-C) reorders subcarriers so that the
zero-frequency bin is in the middle.

Readings taken where the paper is silent: unitary FFT scaling, natural
subcarrier order unless fftshift is asked for, normalised MRC, the Gray
labelling of the transmitter in ``synth``, ties sent to the upper level, and
the PN correlation combined over antennas by power with the earliest lag
winning a tie.

Pins: every function here is checked in ``tests/test_oracle_pins.py`` against
closed forms, a library routine or brute force (see that file's docstring).
"""

from __future__ import annotations

import math
from dataclasses import dataclass
from typing import Dict, Optional

import numpy as np

# --------------------------------------------------------------------------
# 1. CP removal
# --------------------------------------------------------------------------


def to_complex(frame: np.ndarray) -> np.ndarray:
    """Interleaved IQ [..., 2] (int16 or float32) -> complex128, exactly."""
    f = np.asarray(frame).astype(np.float64)
    return f[..., 0] + 1j * f[..., 1]


def strip_cp(y: np.ndarray, N: int, cp: int, S: int) -> np.ndarray:
    """y [M][S (N + CP)] -> r [M][S][N]: drop the first CP samples of each
    OFDM symbol (Sec. II-B)."""
    M = y.shape[0]
    return y.reshape(M, S, N + cp)[:, :, cp:]


# --------------------------------------------------------------------------
# 2. FFT (the DFT by its definition)
# --------------------------------------------------------------------------

_DFT_CACHE: Dict[int, np.ndarray] = {}


def dft_matrix(N: int) -> np.ndarray:
    """W[n, k] = exp(-2j pi (n k mod N) / N) / sqrt(N), the unitary DFT."""
    W = _DFT_CACHE.get(N)
    if W is None:
        n = np.arange(N, dtype=np.int64)
        nk = np.outer(n, n) % N
        W = np.exp(-2j * np.pi * nk / N) / math.sqrt(N)
        _DFT_CACHE[N] = W
    return W


def dft(r: np.ndarray) -> np.ndarray:
    """Unitary forward DFT along the last axis (Sec. II-C, batched over all
    antennas and symbols)."""
    return np.asarray(r, dtype=np.complex128) @ dft_matrix(r.shape[-1])


# --------------------------------------------------------------------------
# 3. Least Squares channel estimation
# --------------------------------------------------------------------------


def ls_estimate(Y_pilot: np.ndarray, X_pilot: np.ndarray) -> np.ndarray:
    """H[m, k] = Y_p[m, k] conj(X_p[k]) / |X_p[k]|^2 (block-type LS, Sec. II-C)."""
    X = np.asarray(X_pilot, dtype=np.complex128)
    return Y_pilot * np.conj(X) / (np.abs(X) ** 2)


# --------------------------------------------------------------------------
# 4. Maximal Ratio Combining
# --------------------------------------------------------------------------


def channel_energy(H: np.ndarray) -> np.ndarray:
    """E[k] = sum_m |H[m, k]|^2, the MRC normaliser formed during estimation."""
    return np.sum(np.abs(H) ** 2, axis=0)


def mrc(H: np.ndarray, Y_data: np.ndarray):
    """z[d, k] = sum_m conj(H[m, k]) Y[m, d, k] / E[k] (Sec. II-C).

    Returns (z [D][N], E [N], bad) where ``bad`` is True when some E[k] is zero
    or not finite; those subcarriers get z = 0.
    """
    E = channel_energy(H)
    num = np.einsum("mk,mdk->dk", np.conj(H), Y_data)
    ok = np.isfinite(E) & (E > 0)
    z = np.zeros_like(num)
    z[:, ok] = num[:, ok] / E[ok]
    return z, E, bool(not np.all(ok))


# --------------------------------------------------------------------------
# 4'. Antenna-split MRC (the distributed receiver of Sec. IV)
# --------------------------------------------------------------------------


def mrc_partial(H: np.ndarray, Y_data: np.ndarray):
    """Partial MRC sums of one shard of antennas (H [m][N], Y_data [m][D][N]).

    P[d, k] = sum over the shard of conj(H[m, k]) Y[m, d, k] and
    E[k] = sum over the shard of |H[m, k]|^2: the two sums of step 4 restricted
    to the shard's antennas.  Adding the partials of a partition of the
    antennas gives the sums of the whole array.
    """
    return np.einsum("mk,mdk->dk", np.conj(H), Y_data), channel_energy(H)


def mrc_combine(P_parts, E_parts):
    """z from shard partials (lists of P [D][N] and E [N]), added in list
    order; zero or non-finite energy gives z = 0 and the flag, as in mrc()."""
    P = np.zeros_like(np.asarray(P_parts[0], np.complex128))
    E = np.zeros(np.asarray(E_parts[0]).shape, np.float64)
    for Pg, Eg in zip(P_parts, E_parts):
        P = P + Pg
        E = E + Eg
    ok = np.isfinite(E) & (E > 0)
    z = np.zeros_like(P)
    z[:, ok] = P[:, ok] / E[ok]
    return z, E, bool(not np.all(ok))


# --------------------------------------------------------------------------
# 5. Gray QAM hard decision
# --------------------------------------------------------------------------


def qam_axis(Q: int):
    """(levels per axis L, amplitude unit A, bits per axis w, axes)."""
    if Q == 2:
        return 2, 1.0, 1, 1
    L = int(round(math.sqrt(Q)))
    assert L * L == Q and L >= 2 and (L & (L - 1)) == 0, Q
    return L, 1.0 / math.sqrt(2.0 * (Q - 1) / 3.0), int(math.log2(L)), 2


def thresholds(Q: int) -> np.ndarray:
    """Decision boundaries of one axis: (2 b - L) A for b = 1 .. L-1."""
    L, A, _, _ = qam_axis(Q)
    return np.array([(2 * b - L) * A for b in range(1, L)], dtype=np.float64)


def slice_axis(v: np.ndarray, Q: int, dtype=np.float64):
    """Level index of each value and its distance to the nearest boundary.

    The level is the number of boundaries at or below ``v`` (a value exactly on
    a boundary goes to the upper level).  ``dtype`` chooses the precision the
    comparison is made in: float64 for the oracle's own decisions, float32 to
    take the decision in the precision of a float32 receiver.
    """
    th = thresholds(Q).astype(dtype)
    vv = np.asarray(v).astype(dtype)
    lvl = np.zeros(vv.shape, dtype=np.int64)
    for t in th:
        lvl += (vv >= t)
    dist = np.min(np.abs(np.asarray(v, np.float64)[..., None]
                         - thresholds(Q)), axis=-1)
    return lvl, dist


def gray_bits(level: np.ndarray, w: int) -> np.ndarray:
    """Gray word level ^ (level >> 1), as w bits MSB-first -> [..., w]."""
    g = level ^ (level >> 1)
    return np.stack([(g >> (w - 1 - j)) & 1 for j in range(w)],
                    axis=-1).astype(np.uint8)


def demap(z: np.ndarray, Q: int, dtype=np.float64):
    """Hard bits [..., q] (I-axis bits first) and decision margin [...]."""
    L, A, w, axes = qam_axis(Q)
    li, di = slice_axis(np.real(z), Q, dtype)
    if axes == 1:
        return gray_bits(li, w), di
    lq, dq = slice_axis(np.imag(z), Q, dtype)
    return (np.concatenate([gray_bits(li, w), gray_bits(lq, w)], axis=-1),
            np.minimum(di, dq))


def pack_bits(bits: np.ndarray) -> np.ndarray:
    """bits [F][...] -> bytes [F][ceil(n / 8)], bit t of a frame at bit
    (7 - t % 8) of byte t / 8 (MSB-first)."""
    F = bits.shape[0]
    flat = bits.reshape(F, -1)
    return np.packbits(flat, axis=-1, bitorder="big")


# --------------------------------------------------------------------------
# 0. Packet detection and output order (Sec. II-B, Sec. II-C)
# --------------------------------------------------------------------------


def pn_metric(capture: np.ndarray, pn: np.ndarray, window: int) -> np.ndarray:
    """Correlation of every antenna's samples with the known PN sequence,
    combined over antennas by power (Sec. II-B: the received signal is
    correlated with the PN sequence to find the start of the packet):
    metric[tau] = sum_m |sum_n conj(pn[n]) y[m, tau + n]|^2, tau < window."""
    y = np.asarray(capture, np.complex128)
    p = np.conj(np.asarray(pn, np.complex128))
    L = p.shape[0]
    metric = np.zeros(window)
    for tau in range(window):
        c = y[:, tau:tau + L] @ p
        metric[tau] = np.sum(np.abs(c) ** 2)
    return metric


def pn_sync(capture: np.ndarray, pn: np.ndarray, window: int):
    """(offset of the preamble = first tau of the largest metric, metric)."""
    metric = pn_metric(capture, pn, window)
    return int(np.argmax(metric)), metric


def extract_frame(capture: np.ndarray, start: int, T: int) -> np.ndarray:
    """The T samples of each antenna row from ``start`` (interleaved IQ kept)."""
    return np.asarray(capture)[:, start:start + T]


def fftshift_rows(x: np.ndarray) -> np.ndarray:
    """Subcarrier order of the paper's output (Sec. II-C, fftshift): the
    zero-frequency bin moves to the middle of the last axis."""
    return np.fft.fftshift(x, axes=-1)


# --------------------------------------------------------------------------
# The whole receiver
# --------------------------------------------------------------------------


@dataclass
class Result:
    Y: np.ndarray        # [F][M][S][N] FFT outputs
    H: np.ndarray        # [F][M][N]   LS estimate
    E: np.ndarray        # [F][N]      channel energy
    z: np.ndarray        # [F][D][N]   equalised, combined symbols
    bits: np.ndarray     # [F][D][N][q]
    margin: np.ndarray   # [F][D][N]
    bad: np.ndarray      # [F] zero-energy flag


def data_symbols(S: int, pilot_idx: int):
    return [s for s in range(S) if s != pilot_idx]


def receive(frames: np.ndarray, N: int, cp: int, S: int, pilot_idx: int,
            Q: int, pilot: np.ndarray, H_given: Optional[np.ndarray] = None,
            keep_Y: bool = True) -> Result:
    """Run the receiver on frames [F][M][S (N + CP)][2].

    ``H_given`` [F][M][N] replaces the LS estimate in the combiner (the
    demodulate-only path).
    """
    F, M = frames.shape[0], frames.shape[1]
    ds = data_symbols(S, pilot_idx)
    D = len(ds)
    q = int(round(math.log2(Q)))
    outY = np.empty((F, M, S, N), np.complex128) if keep_Y else None
    outH = np.empty((F, M, N), np.complex128)
    outE = np.empty((F, N))
    outz = np.empty((F, D, N), np.complex128)
    outb = np.empty((F, D, N, q), np.uint8)
    outm = np.empty((F, D, N))
    bad = np.zeros(F, dtype=bool)
    for f in range(F):
        r = strip_cp(to_complex(frames[f]), N, cp, S)
        Y = dft(r)
        H = ls_estimate(Y[:, pilot_idx, :], pilot) if H_given is None \
            else np.asarray(H_given[f], np.complex128)
        z, E, b = mrc(H, Y[:, ds, :])
        bits, margin = demap(z, Q)
        if keep_Y:
            outY[f] = Y
        outH[f], outE[f], outz[f], outb[f], outm[f], bad[f] = H, E, z, bits, margin, b
    return Result(outY, outH, outE, outz, outb, outm, bad)
