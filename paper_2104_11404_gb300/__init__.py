"""GB300-native Lagrangian hydrodynamics full-order step (arXiv 2104.11404).

The compute path is the CUDA library built from csrc/ (C ABI in
include/lagh.h); `lagh` is its thin ctypes binding and `hydro.Hydro` a
convenience wrapper.  `workloads` holds the seeded synthetic problem set-ups.
"""
