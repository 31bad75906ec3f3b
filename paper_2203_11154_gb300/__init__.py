"""GB300-native ParaDIAG step with the additive element-wise Vanka multigrid.

The compute path is the C-ABI library built from `csrc/` (libparadiag.so); the
Python side is a thin ctypes binding (`api`) that marshals torch tensors into
pointers.  Importing this package loads nothing: `api` loads the library on first
use and raises if it is missing.
"""
