"""RFR (Real-Factors-Recombination) integer polynomial factorisation on B300.

Thin Python binding over the C ABI of ``librfr.so`` (``include/rfr.h`` and
``include/rfr_stages.h``): argument marshalling only.  Every step of the
factorisation runs in the library's CUDA kernels; there is no CPU fallback,
and importing the binding without the built library raises.

    from paper_2410_15880_b300 import Context
    with Context() as ctx:
        res = ctx.factor([1, 0, -10, 0, 1])     # ascending coefficients, monic
        res.factors                               # [[1, 0, -10, 0, 1]]
"""
from ._native import (  # noqa: F401
    RFR_OK, RFR_PENDING, RFRError, Context, PendingBatch, Result, GeneralResult, lib, status_name, squarefree,
    stage_validate, stage_roots, stage_weights, stage_enumerate, stage_match, stage_lowlist, stage_splat, stage_splat_match, stage_prune,
    stage_verify,
    match_workspace_bytes, PLAN_DTYPE, RFR_MAX_DEGREE, RFR_LDC,
    RFR_ROOTS_FP64, RFR_ROOTS_FP32_BULK, RFR_MATCH_AUTO, RFR_MATCH_TABLES, RFR_MATCH_SPLAT, RFR_MATCH_PRUNE,
)
