"""perm(A) mod 3 over F3 on one GB300 (arXiv 2407.20205).

The compute path is the CUDA library ``libperm_f3.so`` (built from ``csrc/``)
behind the C ABI declared in ``include/perm_f3.h``; ``binding`` is the thin
ctypes layer over it.  Importing the package itself loads nothing; the first
use of a binding name loads the library and raises if it is missing.
"""
from __future__ import annotations

import importlib

__all__ = ["binding", "inputs"]


def __getattr__(name):
    if name in ("binding", "inputs", "serve", "build"):
        return importlib.import_module(f"{__name__}.{name}")
    if name.startswith("__"):
        raise AttributeError(name)
    binding = importlib.import_module(f"{__name__}.binding")
    if hasattr(binding, name):
        return getattr(binding, name)
    raise AttributeError(name)
