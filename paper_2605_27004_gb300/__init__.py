"""Anisotropic-equilibrium BGK lattice Boltzmann on GB300 (sm_103a).

The compute path is the CUDA library ``liblbm.so`` (C ABI declared in ``include/lbm.h``);
:mod:`paper_2605_27004_gb300.lbm` is its thin ctypes binding. Importing this package does not
load the library; the first use of :mod:`.lbm` does, and fails loudly if it is missing.
"""
__all__ = ["inputs", "lbm"]
