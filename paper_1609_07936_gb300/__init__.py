"""GB300 library for SAIL, annealing inversion of the Laplace transform (arXiv:1609.07936).

The computation lives in libsail.so (CUDA C++ for sm_103a, C ABI in
include/sail.h); this package is its ctypes binding.  There is no CPU path:
using the binding without a CUDA device or without the built library raises.
"""
from ._capi import (PREC_FP32, PREC_FP64, RESYNC_FP32, RESYNC_FP64, RESYNC_TENSOR, RESYNC_TENSOR_BF16,  # noqa: F401
                    SCHEDULE_GEOMETRIC,
                    SCHEDULE_SELF_COOLING, Batch, Params, Sail, SailError, Server, load, philox, workspace_size)
from .sharded import CudaShard, LocalComm, ShardedAnneal, TorchComm  # noqa: F401,E402
