"""GB300-native Ehrenfest-regularised lattice Boltzmann library.

The compute path is the C-ABI shared library ``liblbm.so`` (hand-written
sm_103a CUDA, declared in ``include/lbm.h``).  ``lbm`` is its thin ctypes
binding; ``inputs`` holds the seeded synthetic workloads; ``strouhal`` is
the host-side shedding-frequency estimator of Sec. 4.2.1.

Importing the package does not load the CUDA library; ``lbm.load()`` does,
and raises if the library is missing or cannot be loaded.
"""
__all__ = ["lbm", "inputs", "strouhal"]
