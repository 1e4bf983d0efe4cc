"""GB300 (sm_103a) library for the ternary 2f1s phase-field lattice Boltzmann step.

The compute path is the CUDA library ``_build/liblbm_gb300.so`` (C ABI in
``include/lbm.h``); ``paper_2311_05091_gb300._lbm`` is its ctypes binding.
Build with ``paper_2311_05091_gb300.build.build()``.  Importing the package
neither loads the library nor touches a GPU.
"""
from .build import LIB, build  # noqa: F401
