"""FP64 CPU oracle of the LS/MRC receiver.

TEST INFRASTRUCTURE: only the tests, the smoke check of ``__graft_entry__``
and the CPU baseline legs of ``bench.py`` may use it.  It shares no code with
the CUDA library.
"""

from .lsas_oracle import (Result, receive, strip_cp, dft, dft_matrix,
                          ls_estimate, channel_energy, mrc, mrc_partial,
                          mrc_combine, demap, slice_axis,
                          thresholds, qam_axis, gray_bits, pack_bits,
                          to_complex, data_symbols, pn_metric, pn_sync,
                          extract_frame, fftshift_rows)

__all__ = ["Result", "receive", "strip_cp", "dft", "dft_matrix", "ls_estimate",
           "channel_energy", "mrc", "mrc_partial", "mrc_combine", "demap", "slice_axis", "thresholds",
           "qam_axis", "gray_bits", "pack_bits", "to_complex", "data_symbols",
           "pn_metric", "pn_sync", "extract_frame", "fftshift_rows"]
