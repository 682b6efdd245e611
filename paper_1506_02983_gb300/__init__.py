"""GB300-native ECMG_jcg: extrapolation cascadic multigrid with Jacobi-preconditioned CG.

The compute path is the CUDA library ``libecmg.so`` (sources in ``csrc/``) behind the C ABI
declared in ``include/ecmg.h``; ``ecmg.py`` is its ctypes binding. Importing this package
does not load the library; ``paper_1506_02983_gb300.ecmg`` does, and fails loudly when the
library has not been built.
"""
