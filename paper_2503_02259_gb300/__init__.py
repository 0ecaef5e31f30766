"""GB300-native on-the-fly Gaussian-process kernel products and GP training loss.

The compute path is the C-ABI library ``libgp.so`` (hand-written sm_103a CUDA);
this package only marshals arguments into it.  Importing the package does not
load the library; the first call that needs it does, and fails loudly if it is
missing.
"""
__all__ = ["inputs"]
