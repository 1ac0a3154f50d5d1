"""GB300-native (sm_103a) quasi-incompressible phase-field lattice Boltzmann
solver (Yang & Guo, arXiv 1507.03521), D2Q9.

The compute path is the C-ABI library ``liblbm.so`` (hand-written CUDA,
declared in ``include/lbm.h``); ``paper_1507_03521_gb300.lbm`` is its thin
ctypes binding.  Importing this package does not load the library.
"""
__all__ = ["lbm", "workloads"]
