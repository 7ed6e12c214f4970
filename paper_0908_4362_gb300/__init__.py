"""GB300-native relaxing-TVD ideal-MHD solver (arXiv:0908.4362, Sects. 3-4).

The compute path is the CUDA library built from ``csrc/`` for sm_103a and reached through
the C ABI declared in ``include/mhd.h``.  Importing this package does not load the library;
``paper_0908_4362_gb300.mhd`` does, and fails loudly if it has not been built.
"""

__all__ = ["inputs"]
