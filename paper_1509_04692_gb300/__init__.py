"""GB300-native checkerboard hard-particle Metropolis Monte Carlo (HPMC).

The compute path is the CUDA library ``libhpmc.so`` built from ``csrc/`` and
reached through the C ABI declared in ``include/hpmc.h``; ``hpmc`` is the thin
ctypes binding (``from paper_1509_04692_gb300 import hpmc``).  Importing the
package itself loads nothing; ``inputs`` (the seeded synthetic
configurations) imports without the CUDA library.
"""
