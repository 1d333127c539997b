"""GB300-native COPSE secure decision-forest inference.

The CUDA library and its C-ABI live in ``csrc/``; ``copse`` is the thin
ctypes binding (imported on demand so that ``synth`` stays usable without a
built library).
"""
