"""GB300 sparsified algebraic multigrid (Bienz et al., arXiv:1512.04629).

The computation lives in libamg.so (CUDA, sm_103a) behind the C ABI of
include/amg.h; this package is its ctypes binding and build script.
"""
import os as _os

# The server runs each registered hierarchy on its own stream.  CUDA spreads
# streams over CUDA_DEVICE_MAX_CONNECTIONS hardware queues (8 by default), and
# streams that share a queue wait on one another; 32 queues keep the
# hierarchies and the server's copies apart.  Read when the process creates
# its CUDA context, so it takes effect only if that happens after this import;
# a value the user set is kept.
_os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

from .amg import (  # noqa: F401,E402
    OK, ERR_INVALID, ERR_OOM, ERR_CUDA, NOT_CONVERGED, DIVERGED, BREAKDOWN, TIMEOUT, REJECTED,
    AmgError, Hierarchy, Matrix, Server, SolveInfo, default_options, device_bytes, kernel_launches, lib,
    debug_fail_allocation, halo_plan,
    METHOD_SPARSE, METHOD_HYBRID, METHOD_NONGALERKIN, LUMP_DIAG, LUMP_STRONG, KRYLOV_CG, KRYLOV_GMRES,
    PREC_FP64, PREC_FP32, PREC_FP32_BF16,
    SPMV_AUTO, SPMV_CSR2, SPMV_CSR4, SPMV_CSR8, SPMV_CSR16, SPMV_CSR32, SPMV_SELL32, SPMV_SELL16, SPMV_SELL8,
    SPMV_CSR1, SPMV_NAMES,
    K_PRE, K_RESTRICT, K_PROLONG, K_POST, K_COARSE, K_AP, K_VEC,
)
