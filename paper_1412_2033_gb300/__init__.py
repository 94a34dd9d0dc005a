"""ghb: guaranteed bounds on homogenized coefficients by the Ga scheme
(Fourier-Galerkin with exact integration) on GB300 (sm_103a).

The computation runs in the CUDA library built from ``csrc/`` (``build.build()``)
behind the C ABI of ``include/ghb.h``; ``ghb`` is its ctypes binding.
"""
from .ghb import (GHB_BOX, GHB_DISK, GHB_DUAL, GHB_ERR_BREAKDOWN, GHB_ERR_CUDA, GHB_ERR_INVALID,  # noqa: F401
                  GHB_ERR_NOT_CONVERGED, GHB_ERR_OOM, GHB_FP32, GHB_FP64, GHB_GANI_DUAL, GHB_GANI_PRIMAL,
                  GHB_MIXED, GHB_OK, GHB_PRIMAL, GHB_SPHERE, TUNE_FIELDS, Batch, Context, GhbError, Options,
                  full_from_half, gram_noalloc, half_from_full, load_library, prolong, tune_get, tune_reset,
                  tune_set)

__all__ = ["Batch", "Context", "gram_noalloc", "prolong", "tune_get", "tune_set", "tune_reset", "TUNE_FIELDS",
           "Options", "GhbError", "load_library", "half_from_full", "full_from_half",
           "GHB_PRIMAL", "GHB_DUAL", "GHB_GANI_PRIMAL", "GHB_GANI_DUAL", "GHB_FP64", "GHB_MIXED", "GHB_FP32",
           "GHB_BOX", "GHB_DISK", "GHB_SPHERE", "GHB_OK", "GHB_ERR_INVALID", "GHB_ERR_OOM",
           "GHB_ERR_NOT_CONVERGED", "GHB_ERR_BREAKDOWN", "GHB_ERR_CUDA"]
