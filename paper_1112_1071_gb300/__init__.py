"""GB300-native Monte-Carlo dust continuum radiative transfer (Lucy LTE temperature solve).

The compute path lives in the CUDA shared library ``libhrt`` (C ABI declared in
``include/hrt.h``); ``paper_1112_1071_gb300.hrt`` is the thin ctypes binding over it.
Importing the package does not load the library; ``hrt.load()`` does, and raises if the
library has not been built.
"""
