"""GB300-native PALMAD: discords of every length in [minL, maxL].

The compute path is the CUDA library ``libpalmad.so`` (built from ``csrc/``
for sm_103a); ``palmad`` is its thin ctypes binding.  ``synth`` holds the
seeded workload generators.  Importing this package does not load the CUDA
library; ``palmad.load()`` does, and fails loudly when it is missing.
"""
__all__ = ["synth", "palmad"]
