"""GB300-native grid-hashing KNN (GHN, arXiv 2004.02290).

The compute path lives in a CUDA shared library behind a C ABI
(``include/ghn_knn.h``); ``paper_2004_02290_gb300.knn`` is the thin ctypes
binding over it.  Importing this package loads nothing; the library is loaded
on first use and the binding raises if it is missing.
"""
