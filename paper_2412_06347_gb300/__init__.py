"""Python binding of libmglma, the GB300 (sm_103a) hot path of multigrid
low-mode averaging (arXiv:2412.06347).

Argument marshalling only: every entry point forwards to the C ABI declared
in ``include/mglma.h`` under the same name; all arithmetic runs in the CUDA
kernels of the library.  Arrays may be numpy ``complex128`` arrays (host
memory) or contiguous torch tensors (``complex128`` or ``float64``) on the
context's device; the library detects which.  There is no CPU fallback: if
``libmglma.so`` cannot be loaded or built, importing this package raises.
"""
from __future__ import annotations

from . import _capi
from ._capi import *  # noqa: F401,F403
from ._capi import MglmaError, Context, lib  # noqa: F401

__all__ = [n for n in dir(_capi) if n.startswith("mglma_") or n.startswith("MGLMA_")] + ["Context", "MglmaError"]
