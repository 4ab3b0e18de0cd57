"""GB300 (sm_103a) library for the graph-based S_N transport sweep on curved high-order meshes.

The compute path is libsnsweep.so (CUDA kernels + C ABI, include/snsweep.h); this package is
its Python binding plus a convenience loader for sn_inputs problems.
"""
from ._lib import (Context, Batch, MLP, SnError, sn_predictor_cfg, load, lib, LIB_PATH, EXPORTED, SN_PREC_FP64, SN_PREC_MIXED, SN_PREC_MIXED_DS, SN_PREC_FP64_INV, SN_PREC_DS_INV, SN_LAUNCH_LEVELS, SN_LAUNCH_DATAFLOW,
                   SN_WEIGHT_UNITY, SN_WEIGHT_FACE, SN_WEIGHT_SIGINVFACE, SN_OK, SN_EINVAL, SN_ECUDA, SN_ETIMEOUT,
                   SN_ENOTCONVERGED, SN_EMESH, SN_ESTATE, sn_quadrature_level_symmetric, sn_moment_noalloc)
from .problem import setup_problem

__all__ = ["Context", "Batch", "MLP", "SnError", "sn_predictor_cfg", "load", "lib", "LIB_PATH", "EXPORTED", "setup_problem",
           "SN_PREC_FP64", "SN_PREC_MIXED", "SN_PREC_MIXED_DS", "SN_PREC_FP64_INV", "SN_PREC_DS_INV", "SN_LAUNCH_LEVELS", "SN_LAUNCH_DATAFLOW", "SN_WEIGHT_UNITY", "SN_WEIGHT_FACE", "SN_WEIGHT_SIGINVFACE",
           "SN_OK", "SN_EINVAL", "SN_ECUDA", "SN_ETIMEOUT", "SN_ENOTCONVERGED", "SN_EMESH", "SN_ESTATE",
           "sn_quadrature_level_symmetric", "sn_moment_noalloc"]
