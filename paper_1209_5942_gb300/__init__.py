"""GB300 (sm_103a) twisted-mass Wilson fermion matrix, even-odd CG, forces,
heatbath and HMC after "Lattice QCD based on OpenCL" (arXiv:1209.5942).

The compute path is the CUDA library ``liblqcd.so`` behind the C ABI in
``include/lqcd.h``; :mod:`.lqcd` is its thin ctypes binding and :mod:`.build`
compiles it.  :mod:`.inputs` draws the seeded synthetic fields.
"""
from . import build  # noqa: F401

__all__ = ["build", "lqcd", "inputs"]
