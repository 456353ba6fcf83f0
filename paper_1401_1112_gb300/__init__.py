"""GB300 (sm_103a) per-level implicit diffusion solve.

The compute path is the C-ABI library ``_build/libats.so`` (declared in
``include/ats.h``); ``ats`` is its thin ctypes binding with the same names.
Importing the package does not load the library; ``ats.lib()`` does, and
fails loudly when it is missing.  There is no CPU fallback.
"""
from . import ats  # noqa: F401

__all__ = ["ats"]
