"""B300 (sm_103a) implementation of the periodic MSC-LBM hot path (arxiv 2609.39474).

The compute path is the in-tree CUDA library libmsclbm.so behind the C ABI in include/msclbm.h;
this package only marshals arguments.  Importing the package does not load the library (so that
the build step can run first); ``paper_2609_39474_b300.lattice`` does, and fails loudly if it is
missing.
"""
__all__ = ["build", "lattice"]
