"""GB300-native CHP stabilizer-tableau simulator (arXiv 2507.03092 hot path).

Submodules:
  circuit  -- op record layout and seeded circuit generators (inputs only)
  streams  -- seeded SplitMix64 coin / noise streams (inputs only)
  binding  -- ctypes binding to the CUDA C-ABI library ``libstab.so``
  build    -- compiles the CUDA library for sm_103a

Importing the package loads nothing; ``binding`` loads the CUDA library on
first use and raises if it is missing.
"""
__all__ = ["circuit", "streams", "binding", "build"]
