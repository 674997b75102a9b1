"""GB300 (sm_103a) implementation of the R-SLB time step (Ambrus & Blaga).

The compute path is the CUDA library ``_build/librslb.so`` behind the C ABI of
``include/rslb.h``; this package holds its build script and a thin ctypes
binding with the same names.
"""
from . import build
from ._lib import (FIELDS, MLP, Bjorken, RslbError, Sod, SodBatch, closure_sample,  # noqa: F401
                   closure_step, load, quadrature, restrict)
