"""GB300-native (sm_103a) direct dedispersion of 2-bit filterbank data and the
transient search built on it (Barsdell et al., "Spotting Radio Transients with
the help of GPUs", Sections 2.2-2.3).

The compute path is the CUDA library built from ``csrc/`` behind the C ABI in
``include/dd.h``; this package is its thin Python binding (ctypes) with
PyTorch supplying device memory and streams.
"""
from ._lib import DDError, load as load_library  # noqa: F401
from .batch import Batch, execute_batch  # noqa: F401
from .search import CAND_DTYPE, DEFAULT_WIDTHS, Search  # noqa: F401
from .classifier import Classifier, init_params  # noqa: F401
from .server import Server  # noqa: F401
from .rfi import RfiMask  # noqa: F401
from .dedisp import (KERNEL_AUTO, KERNEL_SIMPLE, KERNEL_TILED, Plan, as_uint32, compute_delays,  # noqa: F401
                     corner_turn, dedisp_status, out_stride, row_bytes)
