"""GB300-native MRT lattice Boltzmann step with Yu and Chai strain-rate routes.

The compute path is the CUDA library liblbm.so (C ABI in include/lbm.h); ``lbm`` is its thin
Python binding.  ``inputs`` generates seeded synthetic fields.  Build with ``build.build()``.
"""
