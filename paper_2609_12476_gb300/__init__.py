"""GB300 (sm_103a) semicoherent NUFFT resampling search (arXiv:2609.12476).

The work happens in libsrs.so (CUDA kernels behind the C ABI in
include/srs.h); this package only loads it and marshals arguments:

    from paper_2609_12476_gb300 import Context, Params
    ctx = Context(0)
    cands, stat_map, report = ctx.search(strain, mc, Params())
"""
from ._capi import (CAND_DTYPE, EXPORTS, SRS_F32, SRS_F64, SRS_MIXED, SRS_PLAIN_FP64, SRS_WEIGHT_AMPLITUDE,
                    SRS_WEIGHT_EQUAL, Context, Params, SrsError, detection_noncentrality, detection_probability,
                    lib, nsigma_threshold, srs_plan)

__all__ = ["CAND_DTYPE", "EXPORTS", "SRS_F32", "SRS_F64", "SRS_MIXED", "SRS_PLAIN_FP64", "SRS_WEIGHT_AMPLITUDE",
           "SRS_WEIGHT_EQUAL", "Context", "Params", "SrsError", "detection_noncentrality", "detection_probability", "lib",
           "nsigma_threshold", "srs_plan"]
