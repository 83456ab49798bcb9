"""GB300-native preconditioned shifted block FOM for Z = r(tA) B ~= e^{tA} B.

The computation runs in the CUDA library ``lib/libexpm_block.so`` (C ABI in
``include/expm_block.h``); this package only marshals arguments.  PyTorch supplies device
memory and streams.  Importing the package does not load the library; the first call does,
and fails loudly if it has not been built.
"""
from .api import Plan, cf_coeffs, colmajor  # noqa: F401

__all__ = ["Plan", "cf_coeffs", "colmajor"]
