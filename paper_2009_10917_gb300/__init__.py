"""GB300-native Benchmark Streaming operations and CG for high-order hex FEM.

The compute path is the C-ABI library ``libbs.so`` (declared in
``include/bs.h``), built from ``csrc/`` for sm_103a.  ``bs`` is its thin
ctypes binding over torch device tensors; ``synth`` draws the seeded inputs.
Importing the package loads nothing: ``bs`` loads the library on first use and
raises if it is missing.
"""
__all__ = ["bs", "synth"]
