"""GB300-native two-body macro-ion PIC step (arXiv 2208.08038).

The compute path is the CUDA library ``csrc/`` behind the C-ABI declared in
``include/bp.h``; ``binding`` wraps it with ctypes.  Importing this package
loads nothing: the shared library is opened on first use of ``binding``.
"""
__all__ = ["binding", "synth"]
