"""GB300-native harmonic surface mapping algorithm (HSMA, arXiv:1806.04801).

The compute path is the CUDA library ``libhsma.so`` (sources in ``csrc/``),
reached through the C ABI declared in ``include/hsma.h``; ``hsma`` is the thin
ctypes binding.  ``inputs`` holds the seeded synthetic workloads, ``sharded``
the host logic of one system split over several GPUs, ``md`` a velocity-Verlet
loop over the update step, and ``build`` the in-tree nvcc build.
"""
__all__ = ["build", "hsma", "inputs", "md", "sharded"]
