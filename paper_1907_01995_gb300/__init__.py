"""GB300 (sm_103a) implementation of RAC-MBADMM (arXiv:1907.01995).

The method runs in the CUDA library built from csrc/ (C-ABI in
include/rac_admm.h); this package holds the build script and the ctypes
front end.
"""
from .api import Handle, assembly, batch, solve  # noqa: F401
