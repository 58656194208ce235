"""Seeded channel-estimation pairs in the LS domain (input data only).

A row is one antenna's channel over N subcarriers: the N-point DFT of random
multipath taps (L taps uniform in ``taps_range``, exponential power-delay
profile of ``decay`` dB per tap drawn from ``decay_range``, expected total
power 1), and its LS estimate from a +-1 pilot through a unitary FFT at an
SNR drawn from ``snr_db_range``: H_LS = H + W with W ~ CN(0, sigma^2) per
subcarrier, the exact distribution of the LS error in that setting.
"""

from __future__ import annotations

import numpy as np


def ls_pairs(R: int, N: int, snr_db_range=(0.0, 30.0), taps_range=(4, 16),
             decay_range=(1.0, 3.0), seed: int = 0):
    """(true rows H [R][N], LS rows H_LS [R][N], snr_db [R]), complex128."""
    rng = np.random.default_rng([seed, R, N])
    H = np.empty((R, N), np.complex128)
    Hls = np.empty((R, N), np.complex128)
    snr = np.empty(R)
    for r in range(R):
        L = int(rng.integers(taps_range[0], taps_range[1] + 1))
        d = rng.uniform(*decay_range)
        p = 10.0 ** (-d * np.arange(L) / 10.0)
        p /= p.sum()
        h = (rng.standard_normal(L) + 1j * rng.standard_normal(L)) * np.sqrt(p / 2)
        H[r] = np.fft.fft(h, N)
        snr[r] = rng.uniform(*snr_db_range)
        s2 = 10.0 ** (-snr[r] / 10.0)
        w = (rng.standard_normal(N) + 1j * rng.standard_normal(N)) * np.sqrt(s2 / 2)
        Hls[r] = H[r] + w
    return H, Hls, snr
