"""GB300-native graph neural preconditioner (GNP) + FP64 flexible GMRES.

The compute path lives in the C-ABI library ``libgnp.so`` (hand-written sm_103a CUDA,
sources under ``csrc/``, declarations in ``include/gnp.h``).  ``gnp`` is the thin
ctypes binding with the same entry-point names.  Importing this package does not
load the library; the first binding call does, and fails loudly if it is missing.
"""
__all__ = ["inputs"]
