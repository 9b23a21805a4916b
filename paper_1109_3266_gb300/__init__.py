"""GB300-native Monte Carlo dose engine for kV x-ray imaging (the method of
arXiv:1109.3266, gCTD).

Modules:
  ctd      -- Python binding of the C ABI (include/ctd.h); loads the CUDA library
  inputs   -- seeded synthetic phantoms, spectra, sources and workloads
  build    -- compiles the CUDA library in-tree for sm_103a
Importing the package loads nothing; the CUDA library is loaded on first use.
"""
