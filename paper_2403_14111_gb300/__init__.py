"""GB300 (sm_103a) implementation of HETAL's encrypted matrix products
(DiagABT, DiagATB) and the RNS-CKKS operations beneath them.

The computation lives in libhetal_gb300.so (C ABI: include/hetal.h); the
Python module `hetal` is its binding, `workloads` the seeded synthetic inputs.
"""
