"""GB300-native (sm_103a) Monte-Carlo radiative-transfer step in the style of
CRASH2 / pCRASH2 (arXiv:1101.4127): photon-packet emission, cell-by-cell
transport with exact integer deposition, and the per-cell ionisation network
and temperature update, as hand-written CUDA behind a small C ABI.

Submodules:
  native  -- ctypes binding of libcrash.so (the C ABI in include/crash.h)
  build   -- compiles libcrash.so for sm_103a with nvcc
  inputs  -- seeded synthetic workloads (density fields, sources, spectra)
"""
__all__ = ["native", "build", "inputs"]
