"""GB300-native vectorised multi-chain Hamiltonian Monte Carlo.

The compute path is the CUDA library ``libhmc.so`` (built from ``csrc/``),
reached through the C ABI declared in ``include/hmc.h``; ``hmc.py`` is the thin
ctypes binding with the same names.  Importing this package loads nothing;
``paper_2002_01184_gb300.hmc`` loads the library and raises if it is missing.
"""
__all__ = ["workloads", "hmc", "build"]
