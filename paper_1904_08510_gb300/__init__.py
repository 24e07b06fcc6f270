"""GB300-native batched JFNK solver for the implicit electron / electric-potential
system of the MISDC method (arXiv:1904.08510, Sec. 3.2).

Submodules:
  sdcef     ctypes binding of the C ABI in include/sdcef.h (libsdcef.so)
  build     compiles libsdcef.so for sm_103a
  workload  seeded synthetic inputs
"""
