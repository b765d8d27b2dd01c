"""GB300 Helmholtz domain-decomposition solver with deflated-GMRES subdomain solves.

Python binding of libhdd.so (include/hdd.h).  This module only marshals arguments: every step of
assembly, deflation set-up and the inner/outer solves runs in the library's CUDA kernels.  There
is no CPU fallback; importing works without a GPU, but every call needs the CUDA library and a
device, and raises otherwise.

Device memory and streams come from PyTorch: vectors are complex128 CUDA tensors, the stream is
``torch.cuda.current_stream()`` unless one is given.
"""
from __future__ import annotations

import ctypes as C
import os

from ._binding import (HDDError, SolveParams, SolveStats, lib, lib_path, status_name,  # noqa: F401
                       SYMBOLS)
from .solver import Solver  # noqa: F401

__all__ = ["Solver", "SolveParams", "SolveStats", "HDDError", "lib", "lib_path", "SYMBOLS"]
