"""GB300-native checkerboard Monte Carlo for the 3D Heisenberg spin glass.

The compute path is the C-ABI library ``libhsg.so`` (hand-written CUDA for
sm_103a, declared in ``include/hsg.h``); ``paper_1006_2566_gb300.hsg`` is its
thin ctypes binding.  Importing this package loads nothing; the binding loads
the library on first use and raises if it is missing.
"""
__all__ = ["hsg", "inputs"]
