"""GB300-native Monte Carlo estimator of x = exp(tA) v (Acebron, arXiv 1904.12759).

Continuous-time Markov-chain walkers over the indices of a sparse A (Sec. 3)
carry the multiplicative functional of Theorems 1-2; the CUDA library behind
include/mcx.h runs preparation, walkers and reductions on the GPU.  This
package is the thin Python binding (ctypes) used by the tests and benchmark.
"""
from . import _lib
from ._lib import EXPORTS, MCXError, load

_API = ("Plan", "power_iteration", "expm_multiply", "Batch", "CVBatch", "MLP", "cv_prepare", "cv_targets",
        "cv_coefficients", "gather_rate", "debug_fail_alloc", "debug_pool_usage")
__all__ = ["EXPORTS", "MCXError", "load", *_API]


def __getattr__(name):
    # the torch-facing API is imported lazily so that loading the C library
    # (and checking its exports) does not require a GPU
    if name in _API:
        from . import api

        return getattr(api, name)
    raise AttributeError(name)
