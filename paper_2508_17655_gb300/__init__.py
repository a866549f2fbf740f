"""GB300-native generalized ballistic simulated bifurcation (GbSB).

The compute path is the C-ABI library ``libgsb.so`` (hand-written CUDA for
sm_103a); ``paper_2508_17655_gb300.gsb`` is its thin ctypes binding. Importing
this package loads nothing; the library is loaded on first use of ``gsb``.
"""
__all__ = ["gsb", "inputs"]
