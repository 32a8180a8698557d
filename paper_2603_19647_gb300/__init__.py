"""GB300-native ROM-accelerated SI-DSA for implicit S_N transport.

The compute path is the C-ABI library ``librte.so`` (CUDA for sm_103a plus a C++ host
driver) declared in ``include/rte.h``; ``paper_2603_19647_gb300.rte`` is its thin
ctypes binding.  ``paper_2603_19647_gb300.inputs`` holds the seeded synthetic workload
generators.  Importing this package does not load the library; ``rte.load()`` does, and
raises when it has not been built.
"""
__all__ = ["inputs", "rte"]
