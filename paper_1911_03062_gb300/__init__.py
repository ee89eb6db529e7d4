"""GB300-native npFEM cell-suspension solver (arXiv 1911.03062, Supp. Sec. 2.1).

The compute path lives in the CUDA library ``libnpfem.so`` built from
``csrc/`` (see :mod:`paper_1911_03062_gb300.npfem` for the Python binding).
Importing this package loads nothing; the binding loads the library on first
use and raises if it is missing.
"""
