"""Multi-stage CPR / CPTR3 preconditioned FGMRES for GB300 (sm_103a).

The compute path lives in the CUDA library ``libmss.so`` (``csrc/``) behind the
C-ABI declared in ``include/mss.h``; ``paper_1912_04385_gb300.mss`` is the thin
ctypes binding. Importing this package loads nothing: the library is loaded on
first use of the binding, and a missing library is an error, never a fallback.
"""

__all__ = ["synthetic"]
