"""GB300-native Boltzmann-BGK hot path (Dzanic & Martinelli, arXiv 2308.06196): one explicit SSP-RK3
stage on a discrete velocity grid, as hand-written sm_103a CUDA behind a C ABI (include/bgk.h)."""
from . import _build  # noqa: F401

__all__ = ["bgk", "workloads"]
