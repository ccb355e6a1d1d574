"""GB300 (sm_103a) library for the stabilised Darcy-Boussinesq natural-convection state solve,
its adjoint and the design sensitivities of Pollini, Sigmund, Andreasen & Alexandersen
(arXiv 1904.00182).

All arithmetic runs in ``lib/libnatconv.so`` (CUDA kernels behind the C ABI of
``include/natconv.h``). This module only marshals arguments through ctypes: the names mirror the
C entry points. There is no CPU fallback: importing the package without the built library raises
an ImportError that says how to build it (``python -m paper_1904_00182_gb300.build``).
"""

import ctypes
import os

from . import _abi
from ._abi import (NC_ARITH_DF64, NC_ARITH_FP64, NC_BASIS_FP32, NC_BASIS_FP64,  # noqa: F401
                   NC_OBJ_MEAN_T_HEATED, NC_OBJ_SUPG_COMPLIANCE, NC_BC_TOP, NC_BC_CAVITY,
                   NC_REGION_BOX, NC_REGION_CYLINDER, NC_MGOP_EXACT, NC_MGOP_PICARD,
                   NC_SMOOTH_BLOCK_JACOBI, NC_SMOOTH_ZLINE, NC_FILTER_SPECTRAL, NC_FILTER_CHEBYSHEV,
                   NC_PREC_FP64,
                   NC_PREC_MIXED, NatConvError, Grid, Params, Stats, default_params, footprint_bytes,
                   load_library)
from .problem import Problem  # noqa: F401

__all__ = ["Problem", "Grid", "Params", "Stats", "NatConvError", "default_params", "footprint_bytes",
           "NC_PREC_MIXED", "NC_PREC_FP64", "NC_ARITH_DF64", "NC_ARITH_FP64", "NC_BASIS_FP64", "NC_BASIS_FP32",
           "NC_OBJ_MEAN_T_HEATED", "NC_OBJ_SUPG_COMPLIANCE", "NC_BC_TOP", "NC_BC_CAVITY", "NC_REGION_BOX", "NC_REGION_CYLINDER",
           "NC_MGOP_EXACT", "NC_MGOP_PICARD", "NC_SMOOTH_BLOCK_JACOBI", "NC_SMOOTH_ZLINE", "NC_FILTER_SPECTRAL",
           "NC_FILTER_CHEBYSHEV",
           "library_path"]


def library_path():
    return _abi.LIB_PATH
