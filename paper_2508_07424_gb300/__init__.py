"""GB300-native FFT phase-field-fracture RVE library (effective toughness, arXiv 2508.07424).

The compute path is the CUDA shared library ``libpff_gb300.so`` (sources in ``csrc/``, C ABI in
``include/pff_rve.h``). This package only marshals arguments to it: see ``capi`` for the raw
ctypes bindings (same names as the C functions) and ``rve`` for a small numpy-facing wrapper.
Importing the package does not load the library; the first call does, and it raises if the
library has not been built (there is no fallback).
"""
__all__ = ["capi", "rve", "build"]
