"""GB300-native matrix-free FE Kohn-Sham operator (Y = H X) behind a C ABI.

``fe_ks``   -- ctypes binding of libfe_ks.so (same names as include/fe_ks.h)
``problem`` -- builds the C problem struct from a seeded synthetic workload
``build``   -- compiles the CUDA sources for sm_103a
"""
