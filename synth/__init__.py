"""Seeded synthetic uplink frames for the LS/MRC receiver.

This module is the transmitter and the radio channel, nothing of the receiver:
it draws bits, maps them to Gray QAM, modulates OFDM symbols (unitary inverse
DFT through ``numpy.fft.ifft``), prepends the cyclic prefix, passes the stream
through independent multipath Rayleigh channels per receive antenna, adds
white Gaussian noise and optionally quantises to interleaved int16 IQ (sc16).
Its outputs feed both the CUDA library and the FP64 oracle as plain arrays.

The frame layout follows Sec. II-B of the paper (one channel-estimation symbol,
then QAM data symbols; CP + N samples per symbol, per antenna).  ``generate``
makes aligned frames that start at the first CP sample; ``generate_capture``
(``synth.capture``) makes captures with the PN preamble for packet detection
and a random delay before it.
"""

from .frames import (FrameConfig, FrameBatch, generate, qam_map, gray_levels,
                     CONFIGS, config_by_name)
from .capture import CaptureBatch, generate_capture, pn_sequence, PN_LEN
from .lsdomain import ls_pairs

__all__ = ["FrameConfig", "FrameBatch", "generate", "qam_map", "gray_levels",
           "CONFIGS", "config_by_name", "CaptureBatch", "generate_capture",
           "pn_sequence", "PN_LEN", "ls_pairs"]
