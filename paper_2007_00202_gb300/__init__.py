"""GB300-native butterfly-compressed multifrontal solver (sm_103a CUDA behind a C ABI).

The compute path lives in libmf.so (built from csrc/ by build.py); the Python
side only marshals arguments (mf.py).  There is no CPU fallback.
"""
from .mf import (Handle, MfError, Server, analyze_problem, lib, mf_analyze, mf_options_init,  # noqa: F401
                 MF_LATTICE_EDGE, MF_LATTICE_NODE, MF_PREC_C64, MF_PREC_C128, MF_REFINE_GMRES,
                 MF_REFINE_IR, MF_REFINE_NONE, MF_PROF_NARROW_GEMM, MF_PROF_FRONT_GEMM, MF_ORDER_AUTO,
                 MF_ORDER_HYBRID, MF_ORDER_GRAPH)
