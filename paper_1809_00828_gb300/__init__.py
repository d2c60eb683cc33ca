"""GB300-native finite cell Additive-Schwarz PCG (Jomo et al., arXiv:1809.00828).

Submodules:
  inputs -- seeded synthetic geometries and workloads
  fcm    -- ctypes binding of libfcm.so (the C ABI of include/fcm.h)
  build  -- compiles libfcm.so for sm_103a
"""
