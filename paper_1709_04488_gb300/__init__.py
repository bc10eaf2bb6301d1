"""GB300-native grad-h SPH neighbour loop (GANDALF, arXiv:1709.04488).

The compute path is the CUDA library ``libsph.so`` (C ABI in include/sph.h);
``paper_1709_04488_gb300.sph`` is its ctypes binding.  ``ics`` holds the seeded
initial-condition generators.  Importing the package loads nothing; the
binding loads the library on first use and fails loudly if it is missing.
"""
__all__ = ["sph", "ics", "build"]
