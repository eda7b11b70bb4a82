"""GB300-native micro-continuum multiphase Darcy-Brinkman-Stokes VOF time step.

The compute path is the CUDA library ``libmdbs.so`` (C-ABI declared in
``include/mdbs.h``); :mod:`paper_2003_08374_gb300.mdbs` is its thin ctypes
binding.  Importing this package loads nothing; the binding loads the library
on first use and raises if it is missing.
"""
