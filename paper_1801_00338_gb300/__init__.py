"""GB300-native butterfly counting (arXiv 1801.00338): exact wedge aggregation and the estimators built on it.

The compute path is the CUDA library libbfc.so (C ABI in include/bfc.h), loaded
by :mod:`paper_1801_00338_gb300.bfc`.  Importing this package loads nothing;
the first call into ``bfc`` loads the library and raises if it is missing.
"""
