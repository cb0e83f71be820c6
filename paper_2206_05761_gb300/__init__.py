"""GB300 library for the adaptive Haar-wavelet FV1 shallow-water model
(HWFV1, arXiv 2206.05761): C ABI over hand-written sm_103a CUDA kernels,
with a thin ctypes binding (hwfv1.py) and a convenience wrapper (sim.py)."""
from . import hwfv1  # noqa: F401

__all__ = ["hwfv1"]
