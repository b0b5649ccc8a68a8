"""GB300-native Lagrangian transport hot path (MPTRAC-style, arxiv 2211.12616).

The computation lives in ``libmptrac.so`` (hand-written CUDA for sm_103a behind
the C ABI of ``include/mptrac.h``); this package is its thin ctypes binding.
PyTorch provides device memory and streams only.
"""
from ._native import (Context, DiffParams, MptracError, Particles, Surrogate, advect_masked, colstats,
                      copy_probe, load, philox, surr_features, surr_targets,
                      MPTRAC_BF16, MPTRAC_FP16, MPTRAC_FP32, MAX_NZ, SIGNATURES, LIB_PATH,
                      SURR_KERNEL_TCGEN05, SURR_KERNEL_MMA_SYNC, SURR_KERNEL_WAIT_TEST)

__all__ = ["Context", "DiffParams", "MptracError", "Particles", "Surrogate", "advect_masked", "colstats",
           "copy_probe", "load", "philox", "surr_features", "surr_targets",
           "MPTRAC_FP32", "MPTRAC_BF16", "MPTRAC_FP16", "MAX_NZ", "SIGNATURES", "LIB_PATH",
           "SURR_KERNEL_TCGEN05", "SURR_KERNEL_MMA_SYNC", "SURR_KERNEL_WAIT_TEST"]
