"""GB300 recursive Green's function library (NEGF hot path of NEMO5, arXiv:1510.04686).

The numerical work runs in ``_lib/libnegf.so`` (CUDA, sm_103a), reached through its C ABI
(``include/negf.h``).  This package only marshals torch tensors into that ABI.
"""
from .negf import (  # noqa: F401
    NegfError,
    Device,
    options,
    lead_selfenergy,
    rgf_solve,
    scba_step,
    rgf_adjoint,
    integrate,
    zgemm,
    zinv,
    profile,
    profile_reset,
    profile_read,
    launch_count,
    PROF_TC_GEMM,
    RGFFunction,
    GraphSolve,
    solve_ragged,
    tc_config,
    tc_config_count,
    rgf,
    PROF_SLICE,
    PROF_INV,
    PROF_GJ_PANEL,
    workspace_size,
    library,
    PREC_FP64,
    PREC_MIXED,
    PREC_MIXED_40,
    PREC_MIXED_56,
    PREC_AUTO,
    fp64_fallback_count,
)
