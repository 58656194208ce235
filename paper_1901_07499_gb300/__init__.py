"""GB300-native LS channel estimation and MRC demodulation of uplink OFDM
frames for large-scale antenna receivers (arXiv 1901.07499).

The receiver runs in hand-written sm_103a CUDA kernels behind the C ABI of
``include/lsas.h``; :mod:`.lsas` is its Python binding and :mod:`.build`
compiles the library in-tree (``build.build()``).
"""

from . import build
from .build import LIB

__all__ = ["build", "LIB"]
