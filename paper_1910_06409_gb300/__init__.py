"""GB300 Parseval evaluator of the Generalised Kolmogorov Equation (plane channel).

The compute path is the CUDA library ``libgke.so`` (C ABI in include/gke.h);
``_native`` is its ctypes binding, ``api`` a thin convenience layer over it.
Nothing here imports the CPU oracle.
"""
from ._native import (GKE_NPROF, GKE_NTERM, GKE_PREC_BF16X3, GKE_PREC_F64, PROFILES, TERMS,  # noqa: F401
                      GkeError)

__all__ = ["GKE_NPROF", "GKE_NTERM", "GKE_PREC_BF16X3", "GKE_PREC_F64", "PROFILES", "TERMS", "GkeError"]
