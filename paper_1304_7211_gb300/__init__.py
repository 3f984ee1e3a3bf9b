"""GB300-native Richardson-Lucy deconvolution hot path (Welk & Erler,
"Algorithmic Optimisations for Iterative Deconvolution Methods").

The compute path is the CUDA shared library built from ``csrc/`` behind the C
ABI declared in ``include/rl.h``; :mod:`paper_1304_7211_gb300.rl` is its thin
ctypes binding.  :mod:`paper_1304_7211_gb300.synth` draws seeded synthetic
inputs.  Submodules are imported on demand so that importing the package does
not load the CUDA library.
"""
__all__ = ["rl", "synth"]
