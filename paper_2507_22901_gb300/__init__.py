"""libcvsearch: GB300 (sm_103a) colour-pair search for imperceptible colour
vibration (Hattori and Hiraki, SIGGRAPH Asia 2022 Posters, §2 Methods).

The computation lives in the CUDA library ``_build/libcvsearch.so`` (sources in
``csrc/``, C ABI in ``include/cvsearch.h``); this package only marshals
arguments.  There is no CPU fallback: if the library cannot be loaded, every
entry point raises.
"""
from ._build import build  # noqa: F401
from .binding import (  # noqa: F401
    PAIR_DTYPE, PREC_FP32_RECHECK, PREC_FP64, CapacityTable, Context, CvsError, EmbedTable, Server,
    header_functions, lib,
    signal_bounds,
)

__version__ = "0.1.0"
