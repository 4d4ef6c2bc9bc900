"""GB300 (sm_103a) rasterised Steered Mixture of Experts image regression.

The compute path is the CUDA library ``libsmoe.so`` (C ABI, see
``include/smoe.h``); this package is a thin binding over it.  Importing the
package does not load the library; the first call that needs it does, and
fails loudly if it is missing.
"""
__all__ = ["synth"]
