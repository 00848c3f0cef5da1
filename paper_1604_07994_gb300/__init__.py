"""Decoupled (interface-strain) Stokes operator and all-at-once multigrid for GB300.

The compute path lives in the CUDA shared library built from ``csrc/`` (``libsdx.so``) behind
the C-ABI declared in ``include/sdx.h``; :mod:`.sdx` is the thin ctypes binding with the same
names.  :mod:`.workloads` holds the seeded synthetic problem definitions.
"""
