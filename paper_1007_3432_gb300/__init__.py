"""GB300-native Hybrid Monte Carlo for the Hubbard model (arXiv:1007.3432).

The compute path is the CUDA library ``lib/libhubhmc.so`` (sources in
``csrc/``, C ABI in ``include/hubhmc.h``); :mod:`.binding` marshals arguments
to it.  PyTorch supplies device memory and streams only.
"""
from .binding import (HH_DTYPE_F32, HH_DTYPE_F64, HH_FP64, HH_MIXED, HH_OP_M, HH_OP_MT,  # noqa: F401
                      HH_OP_MTM, Context, HHError, load)
