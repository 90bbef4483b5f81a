"""GB300-native solver for the Newton Jacobians of a two-phase porous-media
model with AMG-based preconditioners (after Bui, Elman and Moulton,
arXiv:1611.00127).

``rsflow`` is the Python binding of the CUDA library (C-ABI in
``include/rsflow.h``); ``inputs`` generates seeded synthetic workloads.
Submodules are imported on demand so that input generation works on machines
without CUDA.
"""

__all__ = ["inputs", "rsflow", "build"]
