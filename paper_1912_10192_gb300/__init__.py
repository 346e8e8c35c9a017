"""GB300-native GRMHD block update (H-AMR method, arXiv 1912.10192).

The compute path is the CUDA library built from csrc/ and exposed through the
C ABI declared in include/hamr.h; `hamr` is its thin ctypes binding.
`workloads` generates seeded synthetic initial states.
"""
