"""GB300-native N-1 contingency screen: base-case-preconditioned CG for the
fast-decoupled power flow of every single-branch outage.

The compute path is the CUDA library ``libgpcg.so`` (C ABI in
``include/gpcg.h``); this package is its thin Python binding.
"""
from .binding import (BATCHED_FP32, BATCHED_FP32_F16, BATCHED_FP64, GPCG, MAX_EXT_ROWS, MAX_TAIL_ROWS,
                      PLAIN_FP64, PRECOND_EXACT,
                      PRECOND_IC0, PRECOND_JACOBI, SCEN_DIVERGED, SCEN_ISLAND_NO_GEN,
                      SCEN_MAXITER, SCEN_OK, SCEN_QLIM_OVERFLOW, GPCGError, default_options,
                      load, mask_words, unpack_mask)

def overload_loss(solver, outages, P, b):
    """Differentiable N-1 overload penalty (see autograd.N1OverloadLoss)."""
    from .autograd import N1OverloadLoss
    return N1OverloadLoss.apply(solver, outages, P, b)


__all__ = ["overload_loss", "MAX_EXT_ROWS", "MAX_TAIL_ROWS", "mask_words", "unpack_mask", "BATCHED_FP32_F16", "GPCG", "GPCGError", "default_options", "load", "PLAIN_FP64", "BATCHED_FP32",
           "BATCHED_FP64", "PRECOND_IC0", "PRECOND_JACOBI", "PRECOND_EXACT", "SCEN_OK",
           "SCEN_MAXITER", "SCEN_DIVERGED", "SCEN_ISLAND_NO_GEN", "SCEN_QLIM_OVERFLOW"]
