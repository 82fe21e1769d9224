"""GB300-native kernel polynomial method (KPM): C-ABI CUDA library + thin binding.

The compute path lives in the CUDA library ``libkpm.so`` built from ``csrc/``;
``kpm`` is its ctypes binding.  ``inputs`` draws the seeded synthetic inputs.
"""
__all__ = ["kpm", "inputs"]
