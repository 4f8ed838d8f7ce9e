"""GB300-native signature-kernel library: batched Goursat-PDE solvers on sm_103a.

The compute path is the C-ABI shared library built from ``csrc/`` (``libsigkernel.so``); this
package only marshals arguments to it.  ``workloads`` holds the seeded input generators.
Importing the package does not load the CUDA library; the first call into ``sigkernel`` does,
and raises if the library is missing (there is no CPU fallback).
"""
from __future__ import annotations

import importlib

__all__ = ["workloads", "sigkernel"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
