"""GB300 (sm_103a) solver for complex-shifted Laplacian systems (K + lambda I) z = f
by MINRES with the absolute-value preconditioner of arXiv 2408.00488.

The compute path is libcsl.so (hand-written CUDA behind the C ABI in
include/csl.h); this package is its ctypes binding plus a torch.autograd
wrapper.  PyTorch supplies device memory and streams only.
"""
from ._binding import (Batch, BREAKDOWN, CSLError, CUDA_ERROR, INVALID_ARG, Info, NOT_CONVERGED, OK,  # noqa: F401
                       Helmholtz, OUT_OF_MEMORY, PREC_BF16X3, PREC_BF16X6, PREC_FP32, PREC_FP64, ParaDiag, Plan,
                       SINGULAR_PRECOND, TIMEOUT, UNSUPPORTED_SIZE, lib, precondition_static, probe_sync_cost,
                       status_string,
                       tune_cache_load, tune_cache_save, version)
from .autograd import CSLSolve, solve  # noqa: F401
