"""GB300-native PSTD quantum-scattering path (arXiv 2403.04053).

The compute runs in libpstd.so (CUDA, sm_103a) behind the C ABI of include/pstd.h;
``paper_2403_04053_gb300.pstd`` is its Python binding and ``inputs`` holds the seeded
workload generators.  Importing the package loads nothing; the binding loads the
library on first use and raises if it is missing.
"""
