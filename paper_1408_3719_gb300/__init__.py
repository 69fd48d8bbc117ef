"""GB300-native ALE ADER-WENO finite volumes with time-accurate local time
stepping on moving unstructured triangles (Boscheri, Dumbser, Zanotti).

The compute path lives in the CUDA shared library built from ``csrc/`` and is
reached through :mod:`paper_1408_3719_gb300.aleweno` (a ctypes binding of the
C ABI declared in ``include/aleweno.h``).  Importing this package does not
load the library; :func:`paper_1408_3719_gb300.aleweno.load` does, and raises
if it is missing.
"""
__all__ = ["workloads"]
