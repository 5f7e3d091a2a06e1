"""GB300-native soft-snake simulator: batched compliant-constraint (Jacobi) solve of
chains of 1D pneumatic actuators, after Gasoto et al., arXiv 1904.02833.

The compute lives in libsnakesim.so (CUDA, sm_103a) behind the C-ABI of
include/snakesim.h; this package is its Python binding.
"""
from ._native import SimError, load  # noqa: F401


def build(force: bool = False) -> str:
    from .build import build as _b
    return _b(force=force)
