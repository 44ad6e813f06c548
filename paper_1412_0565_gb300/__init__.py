"""GB300-native cascadic multigrid (CMG) Fiedler-vector solver (arXiv 1412.0565).

The compute path is the CUDA library ``libcmg.so`` (C-ABI declared in
``include/cmg.h``); :mod:`paper_1412_0565_gb300.cmg` is its thin ctypes binding
and :mod:`paper_1412_0565_gb300.inputs` holds the seeded graph generators.
Importing the package does not load the library; the first call into
:mod:`.cmg` does, and fails loudly when it is missing.
"""
__all__ = ["cmg", "inputs"]
