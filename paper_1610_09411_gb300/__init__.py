"""GB300-native ESCAPE census: exact 3-, 4- and 5-vertex subgraph counts
(Pinar, Seshadhri, Vishal, arXiv 1610.09411) computed by hand-written sm_103a
CUDA kernels behind the C ABI of include/escape.h.

``paper_1610_09411_gb300.escape`` is the thin binding of that ABI; it raises
on import if the compiled library is missing (there is no CPU fallback).
"""
__all__ = ["build", "escape"]
