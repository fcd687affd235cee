"""GB300-native half-precision staggered-grid wave stepping.

The compute path lives in ``libwave.so`` (CUDA, sm_103a) behind the C ABI of
``include/wave.h``; :mod:`paper_2310_00236_gb300.wave` is the thin ctypes
binding with the same names. Importing this package has no side effects; the
binding loads the library on first use and raises if it is missing.
"""
