"""GB300 library for the semi-implicit APFC amplitude step (arXiv:1902.09761).

``apfc``   - ctypes binding of libapfc.so (C ABI in include/apfc.h)
``inputs`` - seeded synthetic initial states
``build``  - compiles libapfc.so for sm_103a
"""
